"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed numbers (Table 1, 7/25), closed forms, brute-force patch sums, dense
solves built here from the definitions, manufactured solutions and invariants.
"""
import json
import os

import numpy as np
import pytest

from oracle import core, lfa

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def laplacian_dense(N, lam=0.0):
    """(A + lam I) as a dense matrix from the 1D second difference (Sec. 1)."""
    h = 1.0 / (N + 1)
    T = 2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    A = (np.kron(np.eye(N), T) + np.kron(T, np.eye(N))) / h ** 2
    return A + lam * np.eye(N * N)


def oracle_matrix(fn, m):
    """Columns fn(e_q) of a linear map on C^m."""
    cols = []
    for q in range(m):
        e = np.zeros(m, complex)
        e[q] = 1.0
        cols.append(fn(e))
    return np.array(cols).T


# ---- eq. (6): a, b, c equal the entries of the inverse 4x4 patch matrix ---------------

@pytest.mark.parametrize("eta", [0.0, 1e-4 + 2e-3j, 0.37 - 1.2j, 37.0 + 12.0j, -0.4 + 0.5j])
def test_vanka_abc_equal_patch_inverse(eta):
    h = 0.125
    # element = 2x2 nodes in cyclic order; L_i: (4+eta)/h^2 diagonal, -1/h^2 between
    # cyclic neighbours (the corners of one cell are 5-point neighbours in a cycle)
    Li = np.zeros((4, 4), complex)
    for k in range(4):
        Li[k, k] = (4.0 + eta) / h ** 2
        Li[k, (k + 1) % 4] = Li[k, (k - 1) % 4] = -1.0 / h ** 2
    inv = np.linalg.inv(Li) / h ** 2
    a, b, c = core.vanka_abc(eta)
    assert abs(inv[0, 0] - a) < 1e-14 * abs(a) + 1e-16
    assert abs(inv[0, 1] - b) < 1e-13 * abs(a) + 1e-16
    assert abs(inv[0, 2] - c) < 1e-13 * abs(a) + 1e-16


# ---- eq. (3) and (6): the smoother matrix is the additive patch sum -------------------

@pytest.mark.parametrize("N,lam", [(3, 5.0 + 2.0j), (7, 120.0 - 40.0j), (5, -30.0 + 10.0j)])
def test_vanka_smoother_is_additive_patch_sum(N, lam):
    h = 1.0 / (N + 1)
    eta = lam * h * h
    Li = np.zeros((4, 4), complex)
    for k in range(4):
        Li[k, k] = (4.0 + eta) / h ** 2
        Li[k, (k + 1) % 4] = Li[k, (k - 1) % 4] = -1.0 / h ** 2
    Linv = np.linalg.inv(Li)
    m = N * N
    M = np.zeros((m, m), complex)
    # cells between node rows p, p+1 and columns q, q+1 of the node grid 0..N+1;
    # interior node (i, j) is node (i+1, j+1); boundary corners are dropped (R_i
    # restricts to the interior corners), W_i = I/4
    for p in range(N + 1):
        for q in range(N + 1):
            corners = [(p, q), (p, q + 1), (p + 1, q + 1), (p + 1, q)]
            idx = [((r - 1) * N + (s - 1)) if 1 <= r <= N and 1 <= s <= N else -1
                   for (r, s) in corners]
            for u in range(4):
                for v in range(4):
                    if idx[u] >= 0 and idx[v] >= 0:
                        M[idx[u], idx[v]] += 0.25 * Linv[u, v]
    # oracle: with z = 0 and b = e_q, one step with omega = 1 gives z = M e_q
    Mo = oracle_matrix(lambda e: core.vanka_smooth(N, lam, 1.0, e.reshape(N, N),
                                                   np.zeros((N, N))).ravel(), m)
    assert np.max(np.abs(Mo - M)) < 1e-13 * np.max(np.abs(M))


def test_vanka_step_is_error_propagation():
    """S_j = I - omega M L_j (Sec. 2): the error after one step is S_j e."""
    N, lam, om = 7, 40.0 + 25.0j, 0.9
    rng = np.random.default_rng(5)
    zs = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    b = core.apply_shifted_laplacian(N, lam, zs)
    z0 = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    z1 = core.vanka_smooth(N, lam, om, b, z0)
    M = oracle_matrix(lambda e: core.vanka_smooth(N, lam, 1.0, e.reshape(N, N),
                                                  np.zeros((N, N))).ravel(), N * N)
    S = np.eye(N * N) - om * M @ laplacian_dense(N, lam)
    assert np.allclose((z1 - zs).ravel(), S @ (z0 - zs).ravel(), rtol=0, atol=1e-12)


def test_jacobi_smoother_matrix():
    N, lam = 5, 3.0 - 7.0j
    h = 1.0 / (N + 1)
    M = oracle_matrix(lambda e: core.jacobi_smooth(N, lam, 1.0, e.reshape(N, N),
                                                   np.zeros((N, N))).ravel(), N * N)
    assert np.allclose(M, np.eye(N * N) * h * h / (4.0 + lam * h * h), atol=1e-16)


# ---- the five-point operator ------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 3, 7])
def test_operator_equals_dense(N):
    lam = 2.5 - 1.5j
    L = oracle_matrix(lambda e: core.apply_shifted_laplacian(N, lam, e.reshape(N, N)).ravel(),
                      N * N)
    assert np.allclose(L, laplacian_dense(N, lam), rtol=1e-14, atol=0)


def test_manufactured_solution_second_order():
    """A sin(pi x) sin(pi y) -> 2 pi^2 sin sin: error of the discrete solve is O(h^2)."""
    lam = 10.0 + 20.0j
    errs = []
    for N in (15, 31, 63):
        h = 1.0 / (N + 1)
        t = h * np.arange(1, N + 1)
        Y, X = np.meshgrid(t, t, indexing="ij")
        zs = np.sin(np.pi * X) * np.sin(np.pi * Y)
        b = (2 * np.pi ** 2 + lam) * zs
        om = lfa.omega_table([lam], N, mode="fixed")[0]
        z, it, rr, _ = core.shifted_solve(N, lam, om, b, tol=1e-13, maxit=60)
        assert rr <= 1e-13
        errs.append(np.max(np.abs(z - zs)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.9 < r2 < 4.1


# ---- transfer operators ---------------------------------------------------------------

def test_prolongation_is_four_times_restriction_transpose():
    Nf = 15
    Nc = 7
    R = oracle_matrix(lambda e: core.restrict_fw(Nf, e.reshape(Nf, Nf)).ravel(), Nf * Nf)
    P = oracle_matrix(lambda e: core.prolong_add(Nf, e.reshape(Nc, Nc),
                                                 np.zeros((Nf, Nf))).ravel(), Nc * Nc)
    assert np.allclose(P, 4.0 * R.T, atol=1e-16)
    assert np.allclose(R.sum(axis=1), 1.0)


def test_transfer_exact_on_piecewise_linear():
    """FW reproduces linear functions at coarse points; linear interpolation reproduces
    the tent function min(x,1-x) min(y,1-y), linear between coarse nodes."""
    Nf = 31
    Nc = 15
    hf = 1.0 / (Nf + 1)
    hc = 2 * hf
    tf = hf * np.arange(1, Nf + 1)
    tc = hc * np.arange(1, Nc + 1)
    Yf, Xf = np.meshgrid(tf, tf, indexing="ij")
    Yc, Xc = np.meshgrid(tc, tc, indexing="ij")
    lin = lambda X, Y: 0.3 + 1.7 * X - 2.2 * Y
    rc = core.restrict_fw(Nf, lin(Xf, Yf))
    assert np.allclose(rc, lin(Xc, Yc), atol=1e-14)
    tent = lambda X, Y: np.minimum(X, 1 - X) * np.minimum(Y, 1 - Y)
    zf = core.prolong_add(Nf, tent(Xc, Yc) + 0j, np.zeros((Nf, Nf)))
    # bilinear, not the product of tents along the diagonal cells: compare with the
    # bilinear interpolant, which equals the tent product where the tent is bilinear
    # on each coarse cell (it is: a product of per-axis piecewise-linear functions)
    assert np.allclose(zf, tent(Xf, Yf), atol=1e-14)


# ---- dense solves ------------------------------------------------------------------------

def test_dense_solve_matches_numpy():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    x = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    assert np.allclose(core.dense_solve(A, x), np.linalg.solve(A, x), rtol=1e-12)


def test_coarse_solve_3x3():
    lam = 7.0 + 3.0j
    rng = np.random.default_rng(4)
    b = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    z = core.coarse_solve(3, lam, b)
    assert np.allclose(z.ravel(), np.linalg.solve(laplacian_dense(3, lam), b.ravel()),
                       rtol=1e-13)


@pytest.mark.parametrize("N", [3, 7, 15])
@pytest.mark.parametrize("cycle", [(1, 1, 1), (2, 1, 0)])
def test_shifted_solve_matches_dense(N, cycle):
    gamma, nu1, nu2 = cycle
    prm = core.mg_params(gamma, nu1, nu2, 3)
    rng = np.random.default_rng(N)
    lams = [1e-3 + 60.0j, 250.0 - 80.0j, 6.5 + 0.0j]
    for lam in lams:
        b = rng.uniform(-1, 1, (N, N)) + 1j * rng.uniform(-1, 1, (N, N))
        om = lfa.omega_table([lam], N, mode="lfa", K=32)[0]
        z, it, rr, hist = core.shifted_solve(N, lam, om, b, tol=1e-14, maxit=80, prm=prm)
        ref = np.linalg.solve(laplacian_dense(N, lam), b.ravel()).reshape(N, N)
        assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
        assert rr <= 1e-14 and hist[0] == 1.0
        assert np.all(np.diff(hist) < 0)


def test_zero_rhs():
    z, it, rr, hist = core.shifted_solve(15, 3.0, [0.96] * 3, np.zeros((15, 15)))
    assert it == 0 and rr == 0.0 and not np.any(z)


# ---- multigrid rate against the LFA prediction ---------------------------------------------

def measured_rate(N, lam, prm, om, cycles=8):
    rng = np.random.default_rng(11)
    b = rng.uniform(-1, 1, (N, N)) + 1j * rng.uniform(-1, 1, (N, N))
    _, it, _, hist = core.shifted_solve(N, lam, om, b, tol=0.0, maxit=cycles, prm=prm)
    return (hist[cycles] / hist[3]) ** (1.0 / (cycles - 3))


def test_two_grid_rate_matches_lfa():
    """Two-grid V(1,1) (coarse problem solved exactly) with omega = 24/25: measured
    asymptotic rate against the LFA rho(2) = 0.116 of Table 1."""
    N = 31
    prm = core.mg_params(1, 1, 1, coarsest_n=15)
    rate = measured_rate(N, 1e-3 + 0.0j, prm, [0.96, 0.96])
    assert 0.07 < rate < 0.13


def test_vcycle_rate_matches_lfa():
    N = 127
    prm = core.mg_params(1, 1, 1, coarsest_n=3)
    om = [0.96] * core.num_levels(N)
    for lam in (0.01, 64.0 + 60.0j):
        rate = measured_rate(N, lam, prm, om)
        assert 0.086 < rate < 0.146


def test_jacobi_two_grid_rate_matches_lfa():
    N = 31
    prm = core.mg_params(1, 1, 1, coarsest_n=15, smoother=1)
    rate = measured_rate(N, 1e-3, prm, [0.8, 0.8])
    assert 0.30 < rate < 0.37


# ---- LFA: Table 1, Theorem 2.1, 7/25 -----------------------------------------------------------

def table1():
    with open(os.path.join(GOLDEN, "table1.json")) as f:
        return json.load(f)


def ex1_first_eigenvalue(n):
    """"The first eigenvalue" of Table 1: the first one numpy returns (Remark 2.1
    says the factors do not depend on the choice)."""
    return np.linalg.eigvals(lfa.ex1_bvm_matrix(n))[0]


@pytest.mark.parametrize("smoother", ["jacobi", "vanka"])
def test_table1_reproduced(smoother):
    g = table1()
    row = g[smoother]
    h = g["h"]
    lam = ex1_first_eigenvalue(g["n"])
    w = row["omega_opt"]
    for nu, want in enumerate(row["rho"], start=1):
        got = lfa.two_grid_factor(w, lam, h, nu, smoother)
        assert round(got, 3) == pytest.approx(want, abs=1e-12), (nu, got)
    assert round(lfa.smoothing_factor(w, lam * h * h, smoother), 3) == pytest.approx(row["mu_opt"])
    # omega minimising rho(1), to the two printed decimals
    ws = np.round(np.arange(w - 0.05, w + 0.0501, 0.01), 2)
    r1 = [lfa.two_grid_factor(x, lam, h, 1, smoother, K=64) for x in ws]
    assert ws[int(np.argmin(r1))] == pytest.approx(w)


def test_table1_uniform_over_eigenvalues():
    """Remark 2.1: the same factors for every eigenvalue of B."""
    g = table1()
    h = g["h"]
    ev = np.linalg.eigvals(lfa.ex1_bvm_matrix(g["n"]))
    for lam in ev[:: 37]:
        got = [round(lfa.two_grid_factor(0.96, lam, h, nu, K=64), 3) for nu in (1, 2)]
        assert got == [0.28, 0.116]


def test_phi0_minimum_is_seven_over_25():
    g = table1()["phi0_min"]
    phi0, _ = lfa.thm21_terms(24.0 / 25.0, 0.0)
    assert phi0 == pytest.approx(7.0 / 25.0, abs=1e-14)
    for w in (0.9, 0.95, 0.955, 0.965, 0.97, 1.0):
        assert lfa.thm21_terms(w, 0.0)[0] > 7.0 / 25.0
    assert g["value"] == pytest.approx(0.28)
    w, mu = lfa.omega_opt(0.0)
    assert w == pytest.approx(24.0 / 25.0, abs=1e-9) and mu == pytest.approx(0.28, abs=1e-12)


def test_theorem21_bound_holds():
    for eta in [1e-3j, 0.01 + 0.05j, 0.2 - 0.3j, 1.0 + 2.0j, 3.0]:
        for w in (0.8, 0.96, 1.1):
            mu = lfa.smoothing_factor(w, eta)
            phi0, phij = lfa.thm21_terms(w, eta)
            assert mu <= phi0 + phij + 1e-14


def test_ex1_eigenvalue_bound():
    """|lam_j| < n + sqrt(n)/sqrt(2) for B of eq. (9) (Example 1)."""
    for n in (16, 64, 256):
        ev = np.linalg.eigvals(lfa.ex1_bvm_matrix(n))
        assert np.max(np.abs(ev)) < n + np.sqrt(n) / np.sqrt(2)
        assert np.min(ev.real) > 0


def test_omega_opt_large_shift_tends_to_one():
    """For |eta| large L~ ~ eta/h^2 and M~ ~ h^2/eta: omega_opt -> 1."""
    w, mu = lfa.omega_opt(625.0 + 10.0j)
    assert abs(w - 1.0) < 0.01 and mu < 0.01


# ---- alpha-circulant diagonalisation and the all-at-once system (1) ------------------------------

def alpha_circulant_B(n, tau, alpha):
    """B = (1/tau)(I - C_alpha): backward Euler, with alpha u_n in place of u_0."""
    C = np.eye(n, k=-1)
    C[0, n - 1] = alpha
    return (np.eye(n) - C) / tau


@pytest.mark.parametrize("n,alpha", [(4, 1e-2), (16, 1e-2), (64, 1e-3)])
def test_alpha_circulant_diagonalises_B(n, alpha):
    tau = 1.0 / n
    lam, V, Vinv = core.alpha_circulant(n, tau, alpha)
    B = alpha_circulant_B(n, tau, alpha)
    assert np.linalg.norm(V @ np.diag(lam) @ Vinv - B) <= 1e-11 * np.linalg.norm(B)
    assert np.linalg.norm(V @ Vinv - np.eye(n)) <= 1e-12 * n
    ev = np.linalg.eigvals(B)
    assert max(np.min(np.abs(ev - l)) for l in lam) < 1e-8 * n
    assert max(np.min(np.abs(lam - e)) for e in ev) < 1e-8 * n
    assert np.all(lam.real > 0)


def kron_system(N, n, tau, alpha):
    return np.kron(alpha_circulant_B(n, tau, alpha), np.eye(N * N)) + \
        np.kron(np.eye(n), laplacian_dense(N).real)


def test_paradiag_matches_dense_kronecker_solve():
    N, n, tau, alpha = 7, 4, 0.25, 1e-2
    rng = np.random.default_rng(8)
    f = rng.uniform(-1, 1, (n, N, N))
    u0 = rng.uniform(-1, 1, (N, N))
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    assert np.allclose(fhat[0], f[0] + u0 / tau) and np.array_equal(fhat[1:], f[1:])
    lam, V, Vinv = core.alpha_circulant(n, tau, alpha)
    om = lfa.omega_table(lam, N, mode="lfa", K=32)
    u, im, iters, relres = core.paradiag_solve(N, lam, V, Vinv, om, fhat, tol=1e-14, maxit=80)
    ref = np.linalg.solve(kron_system(N, n, tau, alpha), fhat.ravel()).reshape(n, N, N)
    assert np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)
    assert im <= 1e-11 * np.max(np.abs(ref))
    assert np.all(relres <= 1e-14)


def test_allatonce_residual_equals_kronecker_product():
    N, n, tau, alpha = 5, 6, 1.0 / 6, 1e-3
    rng = np.random.default_rng(9)
    u = rng.standard_normal((n, N, N))
    fhat = rng.standard_normal((n, N, N))
    rn, fn, r = core.allatonce_residual(N, n, tau, alpha, u, fhat, want_r=True)
    ref = fhat.ravel() - kron_system(N, n, tau, alpha) @ u.ravel()
    assert np.allclose(r.ravel(), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    assert rn == pytest.approx(np.linalg.norm(ref)) and fn == pytest.approx(np.linalg.norm(fhat))


def test_time_transform_definition():
    rng = np.random.default_rng(10)
    n, m = 5, 7
    W = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    x = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    y = core.time_transform(W, x)
    ref = np.array([[sum(W[j, k] * x[k, p] for k in range(n)) for p in range(m)]
                    for j in range(n)])
    assert np.allclose(y, ref, rtol=1e-14)


def test_mg_cycle_levels_and_w_cycle():
    """A W-cycle with the coarsest level solved exactly reduces the error by at least
    the V-cycle's factor on the same problem."""
    N, lam = 31, 5.0 + 40.0j
    rng = np.random.default_rng(12)
    b = rng.uniform(-1, 1, (N, N)) + 1j * rng.uniform(-1, 1, (N, N))
    ref = np.linalg.solve(laplacian_dense(N, lam), b.ravel()).reshape(N, N)
    om = [0.96] * 4
    zv = core.mg_cycle(N, lam, om, b, np.zeros((N, N)), core.mg_params(1, 1, 1, 3))
    zw = core.mg_cycle(N, lam, om, b, np.zeros((N, N)), core.mg_params(2, 1, 1, 3))
    ev, ew = np.linalg.norm(zv - ref), np.linalg.norm(zw - ref)
    assert ew <= ev * 1.001 and ev < 0.2 * np.linalg.norm(ref)


def test_sequential_backward_euler_is_alpha_zero_kronecker_solve():
    """alpha = 0 in eq. (1) is backward Euler stepped in sequence: the oracle's time stepping
    equals the dense Kronecker solve with the lower-bidiagonal B_0, and for a spatial
    eigenmode it equals the scalar recursion u_k = u_{k-1} / (1 + tau mu)."""
    N, n, tau = 7, 4, 0.25
    rng = np.random.default_rng(12)
    f = rng.uniform(-1, 1, (n, N, N))
    u0 = rng.uniform(-1, 1, (N, N))
    u = core.sequential_backward_euler(N, n, tau, f, u0)
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    ref = np.linalg.solve(kron_system(N, n, tau, 0.0), fhat.ravel()).reshape(n, N, N)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)
    h = 1.0 / (N + 1)
    t = h * np.arange(1, N + 1)
    y, x = np.meshgrid(t, t, indexing="ij")
    mode = np.sin(2 * np.pi * x) * np.sin(np.pi * y)
    mu = (4 / h ** 2) * (np.sin(np.pi * h) ** 2 + np.sin(np.pi * h / 2) ** 2)
    u = core.sequential_backward_euler(N, n, tau, np.zeros((n, N, N)), mode, kappa=0.5)
    for k in range(n):
        assert np.allclose(u[k], mode / (1 + 0.5 * tau * mu) ** (k + 1), rtol=1e-12, atol=1e-14)


def test_paradiag2_iteration_contracts_by_alpha():
    """ParaDIAG-II: u <- u + P_alpha^{-1}(fhat - A_0 u) with the alpha-circulant step as
    P_alpha converges to the sequential solution, each step reducing the error by at least
    alpha / (1 - alpha) (for diffusion far more: the wrapped-around error is damped by the
    propagator over the whole window)."""
    N, n, tau, alpha = 7, 8, 1.0 / 8, 0.05
    rng = np.random.default_rng(13)
    f = rng.uniform(-1, 1, (n, N, N))
    u0 = rng.uniform(-1, 1, (N, N))
    useq = core.sequential_backward_euler(N, n, tau, f, u0)
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    lam, V, Vinv = core.alpha_circulant(n, tau, alpha)
    om = lfa.omega_table(lam, N, mode="fixed")
    A0 = kron_system(N, n, tau, 0.0)
    u = np.zeros_like(fhat)
    errs = []
    for _ in range(6):
        r = fhat - (A0 @ u.ravel()).reshape(n, N, N)
        d, _, _, _ = core.paradiag_solve(N, lam, V, Vinv, om, r, tol=1e-14, maxit=100)
        u = u + d
        errs.append(np.linalg.norm(u - useq) / np.linalg.norm(useq))
    bound = alpha / (1 - alpha)
    assert errs[0] <= bound and errs[1] <= bound * errs[0]
    assert errs[3] <= 1e-13


def test_extended_precision_residual():
    """The long-double residual of eq. (1): equal to the FP64 one up to the FP64 rounding of
    the formula, and exact where every term is exactly representable (dyadic data on a grid
    with h = 1/8), checked against integer arithmetic."""
    N, n, tau, alpha = 7, 4, 0.25, 0.5
    rng = np.random.default_rng(14)
    u = rng.integers(-64, 64, (n, N, N)) / 8.0
    fhat = rng.integers(-64, 64, (n, N, N)) / 4.0
    rn, r = core.allatonce_residual_ld(N, n, tau, alpha, u, fhat)
    # exact: fhat - (u_k - c u_{k-1})/tau - 64 (4 u_k - nb), all integers / 8
    U = (u * 8).astype(np.int64)
    Fh = (fhat * 8).astype(np.int64)
    ex = np.zeros_like(U)
    for k in range(n):
        prev = U[k - 1] if k > 0 else U[n - 1]
        c = 1 if k > 0 else 0  # alpha = 1/2 handled below
        nb = np.zeros((N, N), np.int64)
        nb[1:, :] += U[k, :-1, :]
        nb[:-1, :] += U[k, 1:, :]
        nb[:, 1:] += U[k, :, :-1]
        nb[:, :-1] += U[k, :, 1:]
        Bu = 4 * (2 * U[k] - (2 * prev if c else prev))  # (u - c prev)/tau, times 2 for alpha
        ex[k] = 2 * Fh[k] - Bu - 2 * 64 * (4 * U[k] - nb)
    assert np.array_equal(r * 16, ex.astype(float))
    assert rn == pytest.approx(np.linalg.norm(ex / 16.0), rel=1e-14)
    # random data: agrees with the FP64 residual to its rounding
    u = rng.standard_normal((n, N, N))
    fhat = rng.standard_normal((n, N, N))
    rn_ld, r_ld = core.allatonce_residual_ld(N, n, tau, alpha, u, fhat)
    rn64, _, r64 = core.allatonce_residual(N, n, tau, alpha, u, fhat, want_r=True)
    assert np.max(np.abs(r_ld - r64)) <= 1e-13 * np.max(np.abs(r64))


def test_long_double_shifted_residual_exact_on_dyadic_data():
    """core.residual_ld (eq. (2) in long double): exact on dyadic data, where every term is
    an integer multiple of 1/64 and the result is computed by integer arithmetic here; equal
    to the FP64 residual up to its rounding on random data."""
    N = 7
    rng = np.random.default_rng(21)
    lam = complex(3.0, -1.5)
    zr = rng.integers(-64, 64, (N, N)) / 8.0
    zi = rng.integers(-64, 64, (N, N)) / 8.0
    br = rng.integers(-64, 64, (N, N)) / 8.0
    bi = rng.integers(-64, 64, (N, N)) / 8.0
    r = core.residual_ld(N, lam, br + 1j * bi, zr + 1j * zi)
    Zr, Zi = (zr * 8).astype(np.int64), (zi * 8).astype(np.int64)
    Br, Bi = (br * 8).astype(np.int64), (bi * 8).astype(np.int64)

    def nb(Z):
        s = np.zeros_like(Z)
        s[1:, :] += Z[:-1, :]
        s[:-1, :] += Z[1:, :]
        s[:, 1:] += Z[:, :-1]
        s[:, :-1] += Z[:, 1:]
        return s
    ih2 = (N + 1) ** 2
    # lam = 3 - 1.5 i: (lam z) * 16 = 48 z - 24 i z  (times 8 for the dyadic scale)
    ex_r = 2 * Br - (6 * Zr + 3 * Zi) - 2 * ih2 * (4 * Zr - nb(Zr))
    ex_i = 2 * Bi - (6 * Zi - 3 * Zr) - 2 * ih2 * (4 * Zi - nb(Zi))
    assert np.array_equal(r.real * 16, ex_r.astype(float))
    assert np.array_equal(r.imag * 16, ex_i.astype(float))
    z = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    b = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    r_ld = core.residual_ld(N, lam, b, z)
    r64 = core.residual(N, lam, b, z)
    assert np.max(np.abs(r_ld - r64)) <= 1e-13 * np.max(np.abs(r64))
