"""Local Fourier analysis of Sec. 2.1 in numpy.  TEST INFRASTRUCTURE ONLY.

Symbols (Sec. 2.1, the display after eq. (6), and eq. (7)), with c_i = cos(theta_i) and eta = lam h^2:
    h^2 L~        = 4 + eta - 2 c_1 - 2 c_2
    M~_e / h^2    = a + b c_1 + b c_2 + c c_1 c_2          (a, b, c of eq. (6))
    M~_Jacobi/h^2 = 1 / (4 + eta)                          (damped Jacobi, Sec. 3)
    S~            = 1 - omega M~ L~
Smoothing factor (eq. (4)): mu_loc = max over theta in T^H of |S~(theta)|.
Optimal parameter (eq. (5)): omega_opt = argmin over real omega of mu_loc.
Two-grid factor (Sec. 2.1, Table 1): for theta in T^L, the four harmonics
theta + pi*(a1, a2) are coupled by full weighting, linear interpolation and the
coarse operator re-discretised at 2h; rho(nu) = max over T^L of the spectral
radius of S~^nu K~ with K~ = I - P~ (L~_2h)^{-1} R~ L~.

Sampling of T^H (a reading: the paper does not say how it samples): the uniform
grid theta_a = -pi/2 + 2 pi a / K, a = 0..K-1, on each axis, keeping the points
with at least one coordinate in [pi/2, 3 pi/2).  K = 64 for the per-shift omega.
"""
import numpy as np

from . import core


def _abc(eta):
    """a, b, c of eq. (6) via the oracle's closed form."""
    return core.vanka_abc(eta)


def smoother_symbol(c1, c2, eta, smoother="vanka"):
    """h^2 * M~ at cos(theta) = (c1, c2)."""
    if smoother == "vanka":
        a, b, c = _abc(eta)
        return a + b * c1 + b * c2 + c * c1 * c2
    if smoother == "jacobi":
        return np.ones_like(c1 * 1.0, dtype=complex) / (4.0 + eta)
    raise ValueError(smoother)


def operator_symbol(c1, c2, eta):
    """h^2 * L~ at cos(theta) = (c1, c2)."""
    return 4.0 + eta - 2.0 * c1 - 2.0 * c2


def high_grid(K=64):
    """cos values (c1, c2) of the high-frequency sample points of T^H."""
    th = -np.pi / 2 + 2 * np.pi * np.arange(K) / K
    t1, t2 = np.meshgrid(th, th, indexing="ij")
    high = (t1 >= np.pi / 2) | (t2 >= np.pi / 2)
    return np.cos(t1[high]), np.cos(t2[high])


def smoothing_factor(omega, eta, smoother="vanka", K=64):
    """mu_loc(S_j) of eq. (4) on the sampled T^H."""
    c1, c2 = high_grid(K)
    s = smoother_symbol(c1, c2, eta, smoother) * operator_symbol(c1, c2, eta)
    return float(np.max(np.abs(1.0 - omega * s)))


def omega_opt(eta, smoother="vanka", K=64, lo=0.5, hi=1.5, width=1e-12):
    """argmin over omega in [lo, hi] of mu_loc by golden-section search; mu_loc is a
    maximum of |1 - omega s| over the samples, convex in real omega.  Returns
    (omega_opt, mu_opt)."""
    c1, c2 = high_grid(K)
    s = smoother_symbol(c1, c2, eta, smoother) * operator_symbol(c1, c2, eta)

    def mu(w):
        return float(np.max(np.abs(1.0 - w * s)))

    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    x1, x2 = b - g * (b - a), a + g * (b - a)
    f1, f2 = mu(x1), mu(x2)
    while b - a > width:
        if f1 <= f2:
            b, x2, f2 = x2, x1, f1
            x1 = b - g * (b - a)
            f1 = mu(x1)
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + g * (b - a)
            f2 = mu(x2)
    w = 0.5 * (a + b)
    return w, mu(w)


def omega_table(lam, N, coarsest_n=3, mode="lfa", smoother="vanka", K=64):
    """omega per shift and level: mode "fixed" gives 24/25 (Vanka, Sec. 2.1) or 4/5
    (Jacobi, Sec. 3); mode "lfa" gives omega_opt(lam_j h_l^2) of eq. (5)."""
    lam = np.atleast_1d(np.asarray(lam, dtype=complex))
    L = core.num_levels(N, coarsest_n)
    out = np.zeros((lam.size, L))
    for l in range(L):
        Nl = N
        for _ in range(l):
            Nl = (Nl - 1) // 2
        h = 1.0 / (Nl + 1)
        for j, lj in enumerate(lam):
            if mode == "fixed":
                out[j, l] = 24.0 / 25.0 if smoother == "vanka" else 0.8
            else:
                out[j, l] = omega_opt(lj * h * h, smoother, K)[0]
    return out


def _fw_symbol(c1, c2):
    """Full weighting symbol (1 + cos t1)(1 + cos t2)/4; linear interpolation has the
    same symbol for P = 4 R^T."""
    return (1.0 + c1) * (1.0 + c2) / 4.0


def two_grid_factor(omega, lam, h, nu, smoother="vanka", K=128):
    """rho(nu) of the two-grid method (Table 1): max over theta in T^L (uniform
    K x K grid on [-pi/2, pi/2)^2 without theta = 0) of the spectral radius of
    S~^nu K~ on the four harmonics."""
    eta = lam * h * h
    th = -np.pi / 2 + np.pi * np.arange(K) / K
    t1, t2 = np.meshgrid(th, th, indexing="ij")
    keep = ~((t1 == 0.0) & (t2 == 0.0))
    t1, t2 = t1[keep], t2[keep]
    P = t1.size
    shifts = [(0, 0), (1, 0), (0, 1), (1, 1)]
    R = np.zeros((P, 1, 4), complex)
    Lf = np.zeros((P, 4), complex)
    S = np.zeros((P, 4), complex)
    for q, (s1, s2) in enumerate(shifts):
        c1 = np.cos(t1 + np.pi * s1)
        c2 = np.cos(t2 + np.pi * s2)
        R[:, 0, q] = _fw_symbol(c1, c2)
        Lf[:, q] = operator_symbol(c1, c2, eta) / (h * h)
        S[:, q] = 1.0 - omega * smoother_symbol(c1, c2, eta, smoother) * operator_symbol(c1, c2, eta)
    H = 2.0 * h
    Lc = (4.0 + lam * H * H - 2.0 * np.cos(2 * t1) - 2.0 * np.cos(2 * t2)) / (H * H)
    Pm = np.transpose(R, (0, 2, 1))
    Kmat = np.eye(4)[None] - (Pm / Lc[:, None, None]) @ (R * Lf[:, None, :])
    T = (S ** nu)[:, :, None] * Kmat
    ev = np.linalg.eigvals(T)
    return float(np.max(np.abs(ev)))


def ex1_bvm_matrix(n):
    """B of eq. (9) (Example 1, tau = 1/n): central differences in the interior rows,
    first row (0, 1/2, ...), last row (..., -1, 1), all over tau."""
    tau = 1.0 / n
    B = np.zeros((n, n))
    for k in range(n - 1):
        if k > 0:
            B[k, k - 1] = -0.5
        B[k, k + 1] = 0.5
    B[n - 1, n - 2] = -1.0
    B[n - 1, n - 1] = 1.0
    return B / tau


def thm21_terms(omega, eta, K=64):
    """phi_0(omega) and phi_j(omega) of Theorem 2.1, eq. (8), in the h-free
    form: phi_0 = max |1 - omega M~_0 A~|, phi_j = max |omega eta (h^-2 M~_e)|."""
    c1, c2 = high_grid(K)
    m0 = smoother_symbol(c1, c2, 0.0)
    phi0 = np.max(np.abs(1.0 - omega * m0 * operator_symbol(c1, c2, 0.0)))
    phij = np.max(np.abs(omega * eta * smoother_symbol(c1, c2, eta)))
    return float(phi0), float(phij)
