"""Seeded synthetic inputs for the heat-equation ParaDIAG workloads.

This module holds none of the method's arithmetic: it draws the random
right-hand sides, sources, shifts and initial values with numpy's PCG64
(`numpy.random.default_rng(seed)`, draws in the order listed) and samples the
initial value on the grid.  Both the CUDA path (through the tests and the
benchmark) and the oracle take their inputs from here.

Workloads (unit square, homogeneous Dirichlet, N x N interior, h = 1/(N+1)):
  shifted-63     N=63,   n=16 alpha-circulant shifts (tau=1/16, alpha=1e-2);
                 b_j = U(-1,1) + i U(-1,1), real parts of all shifts first, seed 0.
  paradiag-511   as paradiag-1023 on N=511 (arrays of 134 MB, still larger than L2): the
                 smaller case of the same kernels for profiler captures.
  paradiag-511-128  as paradiag-2047 (n=128, tau=1/128) on N=511: the smaller case of the
                 n = 128 kernels for profiler captures.
  paradiag-1023  N=1023, n=64 time steps (tau=1/64, alpha=1e-3);
                 u0 = sin(pi x) sin(pi y), f = U(-1,1) [n][N][N], seed 1.
  paradiag-2047  N=2047, n=128 (tau=1/128, alpha=1e-3); as paradiag-1023.
  uneven-8       8 instances N in {127,255,255,511,511,1023,1023,2047},
                 n in {16,32,32,64,64,64,128,128}; shifts lam = r e^{i phi},
                 log10 r ~ U(0,4), phi ~ U(-pi/2+0.05, pi/2-0.05); complex U(-1,1)
                 right-hand sides, seed 2, instance by instance (r, phi, Re b, Im b).
  adjoint-1023   as paradiag-1023 (seed 1 for f), plus a target u_target = sum of 8
                 modes A_q sin(k_q pi x) sin(l_q pi y), k_q, l_q ~ U{1..8}, A_q ~ N(0,1),
                 seed 3 (drawn k, then l, then A).
  examples       the time matrices of Sec. 3: Example 1's boundary-value B (eq. (9)) and
                 Example 2's quasi-BVM B (eq. (10)), and Example 3's Helmholtz shifts.
Smaller variants of the same recipes serve the parity tests.
"""
import numpy as np

WORKLOADS = {
    "shifted-63": dict(kind="shifted", N=63, n=16, tau=1.0 / 16, alpha=1e-2, seed=0),
    "paradiag-511": dict(kind="paradiag", N=511, n=64, tau=1.0 / 64, alpha=1e-3, seed=1),
    "paradiag-511-128": dict(kind="paradiag", N=511, n=128, tau=1.0 / 128, alpha=1e-3, seed=1),
    "paradiag-1023": dict(kind="paradiag", N=1023, n=64, tau=1.0 / 64, alpha=1e-3, seed=1),
    "paradiag-2047": dict(kind="paradiag", N=2047, n=128, tau=1.0 / 128, alpha=1e-3, seed=1),
    "adjoint-1023": dict(kind="adjoint", N=1023, n=64, tau=1.0 / 64, alpha=1e-3, seed=1,
                         target_seed=3),
    "uneven-8": dict(kind="uneven", Ns=(127, 255, 255, 511, 511, 1023, 1023, 2047),
                     ns=(16, 32, 32, 64, 64, 64, 128, 128), seed=2),
}


def complex_rhs(rng, n, N):
    """[n][N][N] complex, real parts drawn first, then imaginary parts, U(-1,1)."""
    re = rng.uniform(-1.0, 1.0, size=(n, N, N))
    im = rng.uniform(-1.0, 1.0, size=(n, N, N))
    return re + 1j * im


def grid_coords(N):
    """Interior node coordinates (x_j, y_i) = ((j+1)h, (i+1)h) as [N][N] arrays."""
    h = 1.0 / (N + 1)
    t = h * np.arange(1, N + 1)
    y, x = np.meshgrid(t, t, indexing="ij")
    return x, y


def sine_initial_value(N):
    """u0 = sin(pi x) sin(pi y) at the interior nodes."""
    x, y = grid_coords(N)
    return np.sin(np.pi * x) * np.sin(np.pi * y)


def shifted_problem(N=63, n=16, seed=0):
    """Right-hand sides of the shifted-systems workload."""
    rng = np.random.default_rng(seed)
    return complex_rhs(rng, n, N)


def paradiag_problem(N=1023, n=64, seed=1, dtype=np.float64):
    """(f [n][N][N] real, u0 [N][N]) of the heat-equation ParaDIAG workload."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1.0, 1.0, size=(n, N, N)).astype(dtype, copy=False)
    return f, sine_initial_value(N).astype(dtype, copy=False)


def random_shifts(rng, n):
    """lam = r e^{i phi}, log10 r ~ U(0,4), phi ~ U(-pi/2+0.05, pi/2-0.05)."""
    logr = rng.uniform(0.0, 4.0, size=n)
    phi = rng.uniform(-np.pi / 2 + 0.05, np.pi / 2 - 0.05, size=n)
    return (10.0 ** logr) * np.exp(1j * phi)


def uneven_problem(Ns=(127, 255, 255, 511, 511, 1023, 1023, 2047),
                   ns=(16, 32, 32, 64, 64, 64, 128, 128), seed=2):
    """List of (N, lam [n], b [n][N][N]) for the batched uneven workload."""
    rng = np.random.default_rng(seed)
    out = []
    for N, n in zip(Ns, ns):
        lam = random_shifts(rng, n)
        b = complex_rhs(rng, n, N)
        out.append((N, lam, b))
    return out


def sine_modes_target(N, seed=3, modes=8):
    """u_target = sum_q A_q sin(k_q pi x) sin(l_q pi y) at the interior nodes."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 9, size=modes)
    l = rng.integers(1, 9, size=modes)
    A = rng.standard_normal(modes)
    x, y = grid_coords(N)
    out = np.zeros((N, N))
    for q in range(modes):
        out += A[q] * np.sin(k[q] * np.pi * x) * np.sin(l[q] * np.pi * y)
    return out


def bvm_time_matrix(n):
    """Example 1's time matrix (eq. (9)), tau = 1/n: rows 1..n-2 are the central
    difference (-1/2, 0, 1/2), the first row (0, 1/2, 0, ...) (its -1/2 u_0 moves to the
    right-hand side), the last row the backward difference (..., -1, 1); all over tau."""
    B = np.zeros((n, n))
    for k in range(n - 1):
        B[k, k + 1] = 0.5
        if k > 0:
            B[k, k - 1] = -0.5
    B[n - 1, n - 2] = -1.0
    B[n - 1, n - 1] = 1.0
    return B * n


def quasi_bvm_time_matrix(n, beta):
    """Example 2's time matrix (eq. (10)), (n+1) x (n+1), tau = 1/n: 1 on the diagonal,
    -1 below it, 1/beta in the top-right corner, all over tau."""
    B = np.eye(n + 1) - np.eye(n + 1, k=-1)
    B[0, n] = 1.0 / beta
    return B * n


def helmholtz_shifts(h):
    """Example 3's shifts -j^2 (1 - 0.5 i) for j = 1, 2, ... with j h <= 1/2."""
    js = np.arange(1, int(np.floor(0.5 / h + 1e-12)) + 1)
    return -(js.astype(float) ** 2) * (1 - 0.5j)
