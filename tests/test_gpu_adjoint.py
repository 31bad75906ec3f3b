"""Differentiation form: the adjoint gradients of J = 0.5 ||u_n - u_target||^2 with respect to
the source f, the initial value u0 and the diffusion coefficient kappa, checked against a
dense-solve reference gradient and against central finite differences of the GPU
forward solve (bar: 1e-6 relative), in FP64 and in the FP32 + refinement form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_11154_gb300 import adjoint, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dense_operator(N, n, tau, alpha, kappa):
    h = 1.0 / (N + 1)
    T = 2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    A = (np.kron(np.eye(N), T) + np.kron(T, np.eye(N))) / h ** 2
    C = np.eye(n, k=-1)
    C[0, n - 1] = alpha
    B = (np.eye(n) - C) / tau
    return np.kron(B, np.eye(N * N)) + kappa * np.kron(np.eye(n), A), A


def loss_and_grads(step, f, u0, kappa, target):
    fd = torch.from_numpy(f).cuda().requires_grad_(True)
    u0d = torch.from_numpy(u0).cuda().requires_grad_(True)
    kd = torch.tensor(kappa, dtype=torch.float64, device="cuda", requires_grad=True)
    u = step(fd, u0d, kd)
    J = 0.5 * torch.sum((u[-1] - torch.from_numpy(target).cuda()) ** 2)
    J.backward()
    torch.cuda.synchronize()
    return float(J), fd.grad.cpu().numpy(), u0d.grad.cpu().numpy(), float(kd.grad)


def loss_only(step, f, u0, kappa, target):
    with torch.no_grad():
        u = step(torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda(),
                 torch.tensor(kappa, dtype=torch.float64, device="cuda"))
        d = u[-1].cpu().numpy() - target
    return 0.5 * float(np.sum(d * d))


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_matches_dense_reference_gradient(precision):
    N, n, tau, alpha, kappa = 7, 4, 0.25, 1e-2, 0.7
    rng = np.random.default_rng(1)
    f = rng.uniform(-1, 1, (n, N, N))
    u0 = inputs.sine_initial_value(N)
    target = inputs.sine_modes_target(N)
    step = adjoint.HeatStep(N, n, tau, alpha, precision=precision, tol=1e-13, maxit=200,
                            max_refine=30)
    J, gf, gu0, gk = loss_and_grads(step, f, u0, kappa, target)
    Amat, A = dense_operator(N, n, tau, alpha, kappa)
    fhat = f.copy()
    fhat[0] += u0 / tau
    u = np.linalg.solve(Amat, fhat.ravel()).reshape(n, N, N)
    g = np.zeros_like(u)
    g[-1] = u[-1] - target
    w = np.linalg.solve(Amat.T, g.ravel()).reshape(n, N, N)
    Jref = 0.5 * np.sum(g[-1] ** 2)
    gk_ref = -sum(float(w[k].ravel() @ (A @ u[k].ravel())) for k in range(n))
    assert abs(J - Jref) <= 1e-10 * Jref
    assert np.linalg.norm(gf - w) <= 1e-8 * np.linalg.norm(w)
    assert np.linalg.norm(gu0 - w[0] / tau) <= 1e-8 * np.linalg.norm(w[0] / tau)
    assert abs(gk - gk_ref) <= 1e-8 * abs(gk_ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_matches_finite_differences_31(precision):
    """31 x 31 grid, n = 8, alpha-circulant tau = 1/64, alpha = 1e-3 (the differentiation
    workload's check size).  J is quadratic in (f, u0), so central differences along a
    direction are exact up to the solves' errors; in kappa they are Richardson-extrapolated
    (eps and eps/2)."""
    N, n, tau, alpha, kappa = 31, 8, 1.0 / 64, 1e-3, 1.0
    f, u0 = inputs.paradiag_problem(N, n, seed=1)
    target = inputs.sine_modes_target(N, seed=3)
    step = adjoint.HeatStep(N, n, tau, alpha, precision=precision, tol=1e-13, maxit=200,
                            max_refine=40)
    J, gf, gu0, gk = loss_and_grads(step, f, u0, kappa, target)
    rng = np.random.default_rng(2)
    df = rng.standard_normal(f.shape)
    du0 = rng.standard_normal(u0.shape)
    eps = 0.5
    fd_f = (loss_only(step, f + eps * df, u0, kappa, target)
            - loss_only(step, f - eps * df, u0, kappa, target)) / (2 * eps)
    fd_u0 = (loss_only(step, f, u0 + eps * du0, kappa, target)
             - loss_only(step, f, u0 - eps * du0, kappa, target)) / (2 * eps)

    def dk(e):
        return (loss_only(step, f, u0, kappa + e, target) - loss_only(step, f, u0, kappa - e, target)) / (2 * e)

    fd_k = (4 * dk(5e-4) - dk(1e-3)) / 3
    assert abs(fd_f - float(np.sum(gf * df))) <= 1e-6 * abs(fd_f)
    assert abs(fd_u0 - float(np.sum(gu0 * du0))) <= 1e-6 * abs(fd_u0)
    assert abs(fd_k - gk) <= 1e-6 * abs(fd_k)
