"""ParaDIAG-II: the alpha-circulant step as the preconditioner of sequential backward Euler
(eq. (1) with alpha = 0), FP64 outer corrections and the FP32 + refinement form, against
the oracle's sequential time stepping."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_2203_11154_gb300 import api, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N,n,alpha", [(63, 8, 1e-2), (127, 16, 1e-3)])
def test_paradiag2_reaches_sequential_backward_euler(precision, N, n, alpha):
    tau = 1.0 / n
    f, u0 = inputs.paradiag_problem(N, n, seed=6)
    c = api.paradiag2_context(N, n, tau, alpha, precision=precision)
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    out = c.paradiag_solve(u, torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda())
    torch.cuda.synchronize()
    uh = u.cpu().numpy()
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    rn, fn = core.allatonce_residual(N, n, tau, 0.0, uh, fhat)
    assert rn / fn <= 1e-10 and out["relres_allatonce"] <= 1e-10
    assert out["refine_steps"] >= 2
    useq = core.sequential_backward_euler(N, n, tau, f, u0)
    # ||L_0^{-1}|| <= sum_k tau (1 + tau mu_min)^{-k-1} <= 1 / mu_min for the block lower
    # triangular backward-Euler operator, mu_min the smallest eigenvalue of A
    h = 1.0 / (N + 1)
    mu = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    assert np.linalg.norm(uh - useq) <= 1.01 * rn / mu + 1e-13 * np.linalg.norm(useq)
    # the alpha-circulant step alone (one solve) is O(alpha) away from it
    c1 = api.alpha_circulant_context(N, n, tau, alpha, precision=precision)
    u1 = torch.empty_like(u)
    c1.paradiag_solve(u1, torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda())
    torch.cuda.synchronize()
    gap = np.linalg.norm(u1.cpu().numpy() - useq) / np.linalg.norm(useq)
    assert gap > 10 * np.linalg.norm(uh - useq) / np.linalg.norm(useq)
