"""The paradiag workloads at full size, in the configuration bench.py times (FP32 multigrid
inside FP64 refinement, FFT transforms, CUDA graphs on a stream of its own): the 1023^2 x 64
step against the oracle's complete FP64 solve, the 2047^2 x 128 step through the oracle's
FP64 residual of eq. (1)."""
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


def gpu_solve(w):
    N, n, tau, alpha = w["N"], w["n"], w["tau"], w["alpha"]
    f, u0 = inputs.paradiag_problem(N, n, seed=w["seed"])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c = api.alpha_circulant_context(N, n, tau, alpha, precision=1, imag_check=0)
        fd = torch.from_numpy(f).cuda()
        u0d = torch.from_numpy(u0).cuda()
        u = torch.empty_like(fd)
        out = c.paradiag_solve(u, fd, u0d)
    torch.cuda.synchronize()
    uh = u.cpu().numpy()
    c.destroy()
    del fd, u0d, u
    return f, u0, uh, out


def test_paradiag_1023_against_oracle_solve():
    w = inputs.WORKLOADS["paradiag-1023"]
    N, n, tau, alpha = w["N"], w["n"], w["tau"], w["alpha"]
    f, u0, uh, out = gpu_solve(w)
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    rn, fn = core.allatonce_residual(N, n, tau, alpha, uh, fhat)
    assert rn / fn <= 1e-10 and out["relres_allatonce"] <= 1e-10
    lam, V, Vinv = core.alpha_circulant(n, tau, alpha)
    om = lfa.omega_table(lam, N, mode="lfa")
    uo, _, _, _ = core.paradiag_solve(N, lam, V, Vinv, om, fhat, tol=1e-12)
    rno, _ = core.allatonce_residual(N, n, tau, alpha, uo, fhat)
    g = (alpha ** (np.arange(n) / n))[:, None, None]
    assert np.linalg.norm(g * (uh - uo)) / np.linalg.norm(g * uo) < 1e-8
    h = 1.0 / (N + 1)
    mu = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    assert np.linalg.norm(uh - uo) <= alpha ** (-(n - 1) / n) / mu * (rn + rno)


def test_paradiag_2047_residual():
    w = inputs.WORKLOADS["paradiag-2047"]
    N, n, tau, alpha = w["N"], w["n"], w["tau"], w["alpha"]
    f, u0, uh, out = gpu_solve(w)
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    rn, fn = core.allatonce_residual(N, n, tau, alpha, uh, fhat)
    assert rn / fn <= 1e-10
    # the oracle's FP64 evaluation differs from the exact residual by at most its rounding,
    # 8 eps || |fhat| + |B||u| + |A||u| ||, accumulated slice by slice
    h = 1.0 / (N + 1)
    acc = 0.0
    for k in range(n):
        a = np.abs(uh[k])
        nb = np.zeros_like(a)
        nb[1:, :] += a[:-1, :]
        nb[:-1, :] += a[1:, :]
        nb[:, 1:] += a[:, :-1]
        nb[:, :-1] += a[:, 1:]
        prev = np.abs(uh[k - 1]) * (alpha if k == 0 else 1.0)
        t = np.abs(fhat[k]) + (a + prev) / tau + (4 * a + nb) / h ** 2
        acc += float(np.sum(t * t))
    noise = 8 * np.finfo(float).eps * np.sqrt(acc) / fn
    assert abs(out["relres_allatonce"] - rn / fn) <= 1e-3 * rn / fn + noise
