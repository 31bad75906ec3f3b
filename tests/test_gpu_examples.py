"""Sec. 3's examples at the paper's sizes, in its multigrid setting (W(1,0) cycles, coarsest
h0 = 1/8, fixed omega, relative residual 1e-8): Example 1 (BVM B of eq. (9), n = 256,
h = tau = 1/256), Example 2 (quasi-BVM B of eq. (10), beta = 0.01, 257 shifts) and
Example 3 (Helmholtz shifts, h = 1/128).  On a spread of shifts the GPU cycle counts of both
smoothers equal the oracle's, and Vanka needs fewer cycles than damped Jacobi (the paper's
figures are not available, so the counts themselves are unpinned)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core, lfa  # noqa: E402
from paper_2203_11154_gb300 import api, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _shifts(which):
    if which == "example1":
        return 255, np.linalg.eigvals(lfa.ex1_bvm_matrix(256))
    if which == "example2":
        B = np.eye(257) - np.eye(257, k=-1)
        B[0, 256] = 1.0 / 0.01
        return 255, np.linalg.eigvals(B * 256)
    js = np.arange(1, 65)
    return 127, -(js ** 2) * (1 - 0.5j)


@pytest.mark.parametrize("which", ["example1", "example2", "example3"])
def test_example_cycle_counts_match_oracle(which):
    N, lam_all = _shifts(which)
    lam = lam_all[np.linspace(0, lam_all.size - 1, 6).astype(int)]
    n = lam.size
    b = inputs.complex_rhs(np.random.default_rng(11), n, N)
    its = {}
    for sm, name in ((0, "vanka"), (1, "jacobi")):
        cfg = api.config(cycle_gamma=2, nu1=1, nu2=0, coarsest_n=7, omega_mode=0, tol=1e-8,
                         maxit=1000, precision=0, smoother=sm)
        c = api.Context(N, n, lam, cfg=cfg)
        z = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
        # damped Jacobi may not converge on Example 3's indefinite shifts: both sides then
        # stop at the same cycle limit
        it, rr = c.shifted_solve_batched(z, torch.from_numpy(b).cuda(), raise_on_noconv=sm == 0)
        om = lfa.omega_table(lam, N, coarsest_n=7, mode="fixed", smoother=name)
        _, ito, rro = core.shifted_solve_batch(N, lam, om, b, tol=1e-8, maxit=1000,
                                               prm=core.mg_params(2, 1, 0, 7, sm))
        assert np.array_equal(it, ito), (name, it, ito)
        conv = ito < 1000
        assert np.all(rr[conv] <= 1e-8)
        if sm == 0:
            assert np.all(conv)
        its[name] = it
        c.destroy()
    assert np.all(its["vanka"] <= its["jacobi"])
