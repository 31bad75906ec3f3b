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


@pytest.mark.parametrize("precision", [1, 0])
def test_adjoint_1023_against_finite_differences(precision):
    """The differentiation workload at full size (1023^2, n = 64, the 8-mode target): the
    adjoint gradients in f and u0 along random directions against central differences of
    the GPU forward solve (exact for the quadratic loss up to the solves' error), bar 1e-6
    relative.  In kappa the reference at 1e-6 is the tangent-linear derivative
    <u_n - target, v_n>, v the forward solve of (B x I + kappa I x A) v = -(I x A) u: at this
    size J is known only to the solves' floor (relres about 4e-12, the FP64 rounding of u
    amplified by 8 kappa/h^2 = 8.4e6), which central differences in kappa divide by the step,
    so they are kept as a check at 1e-5."""
    from paper_2203_11154_gb300 import adjoint
    w = inputs.WORKLOADS["adjoint-1023"]
    N, n, tau, alpha = w["N"], w["n"], w["tau"], w["alpha"]
    f, u0 = inputs.paradiag_problem(N, n, seed=w["seed"])
    target = inputs.sine_modes_target(N, seed=w["target_seed"])
    if precision == 1:
        step = adjoint.HeatStep(N, n, tau, alpha, precision=1, tol=1e-11, max_refine=30)
    else:  # FP64 corrections bring eq. (1) itself to the tolerance (the FP64 residual's
        # own rounding is near 1e-11 at N = 1023)
        step = adjoint.HeatStep(N, n, tau, alpha, precision=0, tol=1e-10, outer_maxit=6)
    tt = torch.from_numpy(target).cuda()

    def loss(fd, u0d, kd):
        u = step(fd, u0d, kd)
        return 0.5 * torch.sum((u[-1] - tt) ** 2)

    fd = torch.from_numpy(f).cuda().requires_grad_(True)
    u0d = torch.from_numpy(u0).cuda().requires_grad_(True)
    kd = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    J = loss(fd, u0d, kd)
    J.backward()
    gf, gu0, gk = fd.grad.detach(), u0d.grad.detach(), float(kd.grad)
    rng = np.random.default_rng(5)
    df = torch.from_numpy(rng.standard_normal(f.shape)).cuda()
    # u0 along the computed gradient: over the unit horizon diffusion damps every initial
    # mode by at least e^{-2 pi^2} ~ 3e-9, so J depends on u0 only weakly; J is quadratic,
    # central differences are exact for any step, and a step of 1e6 along the unit
    # gradient direction moves J far above its rounding
    du0 = gu0 / torch.linalg.vector_norm(gu0)
    f0, u00 = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    one = torch.tensor(1.0, dtype=torch.float64, device="cuda")
    with torch.no_grad():
        eps = 0.5
        fd_f = float(loss(f0 + eps * df, u00, one) - loss(f0 - eps * df, u00, one)) / (2 * eps)
        e0 = 1e6
        fd_u0 = float(loss(f0, u00 + e0 * du0, one) - loss(f0, u00 - e0 * du0, one)) / (2 * e0)

        def dk(e):
            return float(loss(f0, u00, one + e) - loss(f0, u00, one - e)) / (2 * e)

        fd_k = (4 * dk(5e-4) - dk(1e-3)) / 3
        # tangent linear in kappa: A the five-point Laplacian (1/h^2)(4u - sum of the 4
        # neighbours, zero outside), applied to every time step
        h = 1.0 / (N + 1)
        u = step(f0, u00, one)
        au = 4.0 * u
        au[:, 1:, :] -= u[:, :-1, :]
        au[:, :-1, :] -= u[:, 1:, :]
        au[:, :, 1:] -= u[:, :, :-1]
        au[:, :, :-1] -= u[:, :, 1:]
        v = step(-au / h ** 2, torch.zeros_like(u00), one)
        tl_k = float(torch.sum((u[-1] - tt) * v[-1]))
    assert abs(fd_f - float(torch.sum(gf * df))) <= 1e-6 * abs(fd_f)
    assert abs(fd_u0 - float(torch.sum(gu0 * du0))) <= 1e-6 * abs(fd_u0)
    assert abs(tl_k - gk) <= 1e-6 * abs(tl_k)
    assert abs(fd_k - gk) <= 1e-5 * abs(fd_k)
