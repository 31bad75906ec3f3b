"""The time matrices and shifts of the paper's examples (Sec. 3), in the paper's multigrid
setting (W cycles with one pre- and no post-smoothing step, coarsest h0 = 1/8, fixed
omega): the BVM B of Example 1 (eq. (9)), the quasi-BVM B of Example 2 (eq. (10)), the
Helmholtz shifts of Example 3, and the damped-Jacobi comparison, each against the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core, lfa  # noqa: E402
from paper_2203_11154_gb300 import api, inputs  # noqa: E402

PAPER = dict(cycle_gamma=2, nu1=1, nu2=0, coarsest_n=7, omega_mode=0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def qbvm_matrix(n, beta):
    """B of eq. (10), (n+1) x (n+1), tau = 1/n: 1 on the diagonal, -1 below it, 1/beta in
    the top-right corner, all over tau."""
    B = np.eye(n + 1) - np.eye(n + 1, k=-1)
    B[0, n] = 1.0 / beta
    return B * n


def laplacian(N):
    h = 1.0 / (N + 1)
    T = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    I = sp.identity(N)
    return ((sp.kron(I, T) + sp.kron(T, I)) / h ** 2).tocsr()


@pytest.mark.parametrize("which", ["ex1", "ex2"])
def test_paradiag_general_B(which):
    """u of (B kron I + I kron A) u = fhat with a dense B passed alone to paradiag_setup
    (the library diagonalises it); the initial value enters Example 1's central-difference
    first row as u0 / (2 tau).  The oracle diagonalises B with numpy's LAPACK; the two
    eigenvalue orders are matched by value, and the cycle counts per shift (which do not
    depend on how an eigenvector is scaled) must agree."""
    N = 63
    if which == "ex1":
        n = 16
        B = lfa.ex1_bvm_matrix(n)
        c0 = np.zeros(n)
        c0[0] = n / 2.0
    else:
        B = qbvm_matrix(15, 0.01)
        n = B.shape[0]
        c0 = np.zeros(n)
    c = api.dense_B_context(B, N, c0, tol=1e-10, **PAPER)
    f, u0 = inputs.paradiag_problem(N, n, seed=5)
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    out = c.paradiag_solve(u, torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda())
    lam, V = np.linalg.eig(B)
    Vinv = np.linalg.inv(V)
    om = lfa.omega_table(lam, N, coarsest_n=7, mode="fixed")
    fhat = f + c0[:, None, None] * u0[None]
    uo, _, ito, _ = core.paradiag_solve(N, lam, V, Vinv, om, fhat, tol=1e-10,
                                        prm=core.mg_params(2, 1, 0, 7))
    lam_lib = api.pd_diagonalize(B)[0]
    d = np.abs(lam_lib[:, None] - lam[None, :])
    perm = np.argmin(d, axis=1)
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.max(d[np.arange(n), perm]) <= 1e-9 * np.max(np.abs(lam))
    assert np.array_equal(out["iters"], ito[perm])
    assert np.all(out["relres"] <= 1e-10)
    torch.cuda.synchronize()
    uh = u.cpu().numpy()
    condV = np.linalg.cond(V)
    assert np.linalg.norm(uh - uo) <= condV * 1e-12 * np.linalg.norm(uo)
    A = laplacian(N)
    U = uh.reshape(n, -1)
    res = fhat.reshape(n, -1) - B @ U - (A @ U.T).T
    fn = np.linalg.norm(fhat)
    rel = np.linalg.norm(res) / fn
    assert rel <= condV * 1e-10
    # two FP64 evaluations of the residual differ by at most their rounding errors
    Ua = np.abs(U)
    t = np.abs(fhat.reshape(n, -1)) + np.abs(B) @ Ua + (abs(A) @ Ua.T).T
    noise = 8 * np.finfo(float).eps * np.linalg.norm(t) / fn
    assert abs(out["relres_allatonce"] - rel) <= 1e-3 * rel + noise


def test_helmholtz_shifts_example3():
    """lam_j = -j^2 (1 - 0.5 i), j = 1..64 (j h <= 1/2 at h = 1/128): negative real parts,
    outside Theorem 2.1.  The GPU cycles follow the oracle's shift by shift, and the counts
    grow with j (Example 3)."""
    N = 127
    js = np.arange(1, 65)
    lam = -(js ** 2) * (1 - 0.5j)
    n = lam.size
    b = inputs.complex_rhs(np.random.default_rng(3), n, N)
    c = api.Context(N, n, lam, cfg=api.config(tol=1e-8, maxit=300, **PAPER))
    z = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    it, rr = c.shifted_solve_batched(z, torch.from_numpy(b).cuda())
    om = lfa.omega_table(lam, N, coarsest_n=7, mode="fixed")
    zo, ito, rro = core.shifted_solve_batch(N, lam, om, b, tol=1e-8, maxit=300,
                                            prm=core.mg_params(2, 1, 0, 7))
    assert np.array_equal(it, ito)
    assert np.all(rr <= 1e-8)
    torch.cuda.synchronize()
    zh = z.cpu().numpy()
    err = np.linalg.norm((zh - zo).reshape(n, -1), axis=1) / np.linalg.norm(zo.reshape(n, -1), axis=1)
    assert np.max(err) <= 1e-10
    assert it[-1] > it[0]


def test_jacobi_comparator_example1():
    """Damped Jacobi (omega = 4/5) against Vanka (omega = 24/25) on the 128 eigenvalues of
    Example 1's B with tau = h = 1/128: both follow the oracle cycle for cycle, and the
    Vanka smoother needs fewer than half the W cycles (Sec. 3, Table 1)."""
    N, n = 127, 128
    lam = np.linalg.eigvals(lfa.ex1_bvm_matrix(n))
    b = inputs.complex_rhs(np.random.default_rng(4), n, N)
    its = {}
    for sm, name in ((0, "vanka"), (1, "jacobi")):
        c = api.Context(N, n, lam, cfg=api.config(smoother=sm, tol=1e-8, maxit=300, **PAPER))
        z = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
        its[name], rr = c.shifted_solve_batched(z, torch.from_numpy(b).cuda())
        om = lfa.omega_table(lam, N, coarsest_n=7, mode="fixed", smoother=name)
        zo, ito, _ = core.shifted_solve_batch(N, lam, om, b, tol=1e-8, maxit=300,
                                              prm=core.mg_params(2, 1, 0, 7, sm))
        assert np.array_equal(its[name], ito)
        torch.cuda.synchronize()
        zh = z.cpu().numpy()
        assert np.linalg.norm(zh - zo) <= 1e-10 * np.linalg.norm(zo)
        c.destroy()
    assert 2 * np.mean(its["vanka"]) < np.mean(its["jacobi"])
