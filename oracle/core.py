"""ctypes wrapper of the C oracle (oracle.c).  TEST INFRASTRUCTURE ONLY.

All arrays are numpy: complex128 grid vectors [N][N] or [n][N][N], float64 real
vectors.  Every wrapper checks shapes and contiguity and copies nothing it does
not have to.  See oracle.c for the passage each routine follows.
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None


class MGParams(C.Structure):
    """gamma (1 = V, 2 = W), nu1/nu2 smoothing steps, coarsest interior size,
    smoother (0 = additive Vanka eq. (6), 1 = damped Jacobi)."""
    _fields_ = [("gamma", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("coarsest_n", C.c_int), ("smoother", C.c_int)]


def mg_params(gamma=1, nu1=1, nu2=1, coarsest_n=3, smoother=0):
    return MGParams(gamma, nu1, nu2, coarsest_n, smoother)


class _Cplx(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


def _c(z):
    z = complex(z)
    return _Cplx(z.real, z.imag)


_P = C.c_void_p
_I = C.c_int
_D = C.c_double


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "or_apply_shifted_laplacian": (None, [_I, _D, _Cplx, _P, _P]),
            "or_residual": (None, [_I, _D, _Cplx, _P, _P, _P]),
            "or_vanka_abc": (None, [_Cplx, _P, _P, _P]),
            "or_vanka_smooth": (None, [_I, _D, _Cplx, _D, _P, _P]),
            "or_jacobi_smooth": (None, [_I, _D, _Cplx, _D, _P, _P]),
            "or_restrict_fw": (None, [_I, _P, _P]),
            "or_prolong_add": (None, [_I, _P, _P]),
            "or_dense_solve": (_I, [_I, _P, _P]),
            "or_coarse_solve": (_I, [_I, _D, _Cplx, _P, _P]),
            "or_mg_cycle": (_I, [C.POINTER(MGParams), _I, _Cplx, _P, _P, _P]),
            "or_shifted_solve": (_I, [C.POINTER(MGParams), _I, _Cplx, _P, _I, _D, _P, _P,
                                      _P, _P, _P]),
            "or_shifted_solve_batch": (_I, [C.POINTER(MGParams), _I, _I, _P, _P, _I, _I, _D,
                                            _P, _P, _P, _P]),
            "or_alpha_circulant": (None, [_I, _D, _D, _P, _P, _P]),
            "or_assemble_rhs": (None, [_I, _I, _D, _P, _P, _P]),
            "or_time_transform": (None, [_I, C.c_size_t, _P, _P, _P]),
            "or_paradiag_solve": (_I, [C.POINTER(MGParams), _I, _I, _P, _P, _P, _P, _I, _I,
                                       _D, _P, _P, _P, _P, _P]),
            "or_allatonce_residual": (_D, [_I, _I, _D, _D, _P, _P, _P, _P]),
            "or_allatonce_residual_ld": (_D, [_I, _I, _D, _D, _P, _P, _P]),
            "or_residual_ld": (_D, [_I, _D, _Cplx, _P, _P, _P]),
            "or_set_threads": (None, [_I]),
            "or_max_threads": (_I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _cvec(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _rvec(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def num_levels(N, coarsest_n=3):
    """Levels N, (N-1)/2, ... down to the first size <= coarsest_n."""
    L = 1
    while N > coarsest_n:
        N = (N - 1) // 2
        L += 1
    return L


def apply_shifted_laplacian(N, lam, z):
    z = _cvec(z, (N, N))
    out = np.empty_like(z)
    lib().or_apply_shifted_laplacian(N, 1.0 / (N + 1), _c(lam), _ptr(z), _ptr(out))
    return out


def residual(N, lam, b, z):
    b = _cvec(b, (N, N))
    z = _cvec(z, (N, N))
    r = np.empty_like(z)
    lib().or_residual(N, 1.0 / (N + 1), _c(lam), _ptr(b), _ptr(z), _ptr(r))
    return r


def vanka_abc(eta):
    out = [np.zeros(1, np.complex128) for _ in range(3)]
    lib().or_vanka_abc(_c(eta), *[_ptr(o) for o in out])
    return tuple(complex(o[0]) for o in out)


def vanka_smooth(N, lam, omega, b, z):
    b = _cvec(b, (N, N))
    z = _cvec(z, (N, N)).copy()
    lib().or_vanka_smooth(N, 1.0 / (N + 1), _c(lam), float(omega), _ptr(b), _ptr(z))
    return z


def jacobi_smooth(N, lam, omega, b, z):
    b = _cvec(b, (N, N))
    z = _cvec(z, (N, N)).copy()
    lib().or_jacobi_smooth(N, 1.0 / (N + 1), _c(lam), float(omega), _ptr(b), _ptr(z))
    return z


def restrict_fw(Nf, rf):
    rf = _cvec(rf, (Nf, Nf))
    Nc = (Nf - 1) // 2
    rc = np.empty((Nc, Nc), np.complex128)
    lib().or_restrict_fw(Nf, _ptr(rf), _ptr(rc))
    return rc


def prolong_add(Nf, ec, zf):
    Nc = (Nf - 1) // 2
    ec = _cvec(ec, (Nc, Nc))
    zf = _cvec(zf, (Nf, Nf)).copy()
    lib().or_prolong_add(Nf, _ptr(ec), _ptr(zf))
    return zf


def dense_solve(A, x):
    A = _cvec(A).copy()
    x = _cvec(x).copy()
    m = x.shape[0]
    if A.shape != (m, m):
        raise ValueError("A must be m x m")
    rc = lib().or_dense_solve(m, _ptr(A), _ptr(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular pivot")
    return x


def coarse_solve(N, lam, b):
    b = _cvec(b, (N, N))
    z = np.empty_like(b)
    rc = lib().or_coarse_solve(N, 1.0 / (N + 1), _c(lam), _ptr(b), _ptr(z))
    if rc != 0:
        raise np.linalg.LinAlgError("singular coarse matrix")
    return z


def mg_cycle(N, lam, omega_levels, b, z, prm=None):
    prm = prm or mg_params()
    b = _cvec(b, (N, N))
    z = _cvec(z, (N, N)).copy()
    om = _rvec(omega_levels)
    if om.size < num_levels(N, prm.coarsest_n):
        raise ValueError("need one omega per level")
    rc = lib().or_mg_cycle(C.byref(prm), N, _c(lam), _ptr(om), _ptr(b), _ptr(z))
    if rc != 0:
        raise np.linalg.LinAlgError("singular coarse matrix")
    return z


def shifted_solve(N, lam, omega_levels, b, tol=1e-10, maxit=100, prm=None):
    """Returns (z, iters, relres, history of relres after 0..iters cycles)."""
    prm = prm or mg_params()
    b = _cvec(b, (N, N))
    z = np.empty_like(b)
    om = _rvec(omega_levels)
    if om.size < num_levels(N, prm.coarsest_n):
        raise ValueError("need one omega per level")
    it = C.c_int(0)
    rr = C.c_double(0.0)
    hist = np.zeros(maxit + 1)
    rc = lib().or_shifted_solve(C.byref(prm), N, _c(lam), _ptr(om), int(maxit), float(tol),
                                _ptr(b), _ptr(z), C.byref(it), C.byref(rr), _ptr(hist))
    if rc != 0:
        raise np.linalg.LinAlgError("singular coarse matrix")
    return z, it.value, rr.value, hist[: it.value + 1].copy()


def shifted_solve_batch(N, lam, omega, b, tol=1e-10, maxit=100, prm=None):
    """lam: [n] complex; omega: [n][levels]; b: [n][N][N].  Returns (z, iters, relres)."""
    prm = prm or mg_params()
    lam = _cvec(lam)
    n = lam.shape[0]
    b = _cvec(b, (n, N, N))
    om = _rvec(omega)
    levels = om.shape[1]
    if om.shape[0] != n or levels < num_levels(N, prm.coarsest_n):
        raise ValueError("omega must be [n][levels]")
    z = np.empty_like(b)
    iters = np.zeros(n, np.int32)
    relres = np.zeros(n)
    rc = lib().or_shifted_solve_batch(C.byref(prm), N, n, _ptr(lam), _ptr(om), levels,
                                      int(maxit), float(tol), _ptr(b), _ptr(z), _ptr(iters),
                                      _ptr(relres))
    if rc != 0:
        raise np.linalg.LinAlgError("singular coarse matrix")
    return z, iters, relres


def alpha_circulant(n, tau, alpha):
    """Returns (lam [n], V [n][n], Vinv [n][n]) of B = (1/tau)(I - C_alpha)."""
    lam = np.empty(n, np.complex128)
    V = np.empty((n, n), np.complex128)
    Vinv = np.empty((n, n), np.complex128)
    lib().or_alpha_circulant(n, float(tau), float(alpha), _ptr(lam), _ptr(V), _ptr(Vinv))
    return lam, V, Vinv


def assemble_rhs(N, n, tau, f, u0):
    f = _rvec(f, (n, N, N))
    u0 = _rvec(u0, (N, N))
    fhat = np.empty_like(f)
    lib().or_assemble_rhs(N, n, float(tau), _ptr(f), _ptr(u0), _ptr(fhat))
    return fhat


def time_transform(W, x):
    W = _cvec(W)
    n = W.shape[0]
    x = _cvec(x)
    if x.shape[0] != n:
        raise ValueError("x must have n rows")
    m = x.size // n
    y = np.empty_like(x)
    lib().or_time_transform(n, m, _ptr(W), _ptr(x), _ptr(y))
    return y


def paradiag_solve(N, lam, V, Vinv, omega, fhat, tol=1e-10, maxit=100, prm=None):
    """Returns (u real [n][N][N], max|Im|, iters [n], relres [n])."""
    prm = prm or mg_params()
    lam = _cvec(lam)
    n = lam.shape[0]
    V = _cvec(V, (n, n))
    Vinv = _cvec(Vinv, (n, n))
    om = _rvec(omega)
    levels = om.shape[1]
    fhat = _rvec(fhat, (n, N, N))
    u = np.empty_like(fhat)
    im = C.c_double(0.0)
    iters = np.zeros(n, np.int32)
    relres = np.zeros(n)
    rc = lib().or_paradiag_solve(C.byref(prm), N, n, _ptr(lam), _ptr(V), _ptr(Vinv), _ptr(om),
                                 levels, int(maxit), float(tol), _ptr(fhat), _ptr(u),
                                 C.byref(im), _ptr(iters), _ptr(relres))
    if rc != 0:
        raise np.linalg.LinAlgError("singular coarse matrix")
    return u, im.value, iters, relres


def allatonce_residual(N, n, tau, alpha, u, fhat, want_r=False):
    """Returns (||r||_2, ||fhat||_2[, r]) for eq. (1) with the alpha-circulant B."""
    u = _rvec(u, (n, N, N))
    fhat = _rvec(fhat, (n, N, N))
    r = np.empty_like(u) if want_r else None
    fn = C.c_double(0.0)
    rn = lib().or_allatonce_residual(N, n, float(tau), float(alpha), _ptr(u), _ptr(fhat),
                                     _ptr(r) if want_r else None, C.byref(fn))
    return (rn, fn.value, r) if want_r else (rn, fn.value)


def residual_ld(N, lam, b, z):
    """r = b - (A + lam I) z of eq. (2) evaluated in long double and rounded to double at the
    end (a reference below the FP64 rounding of the formula)."""
    b = _cvec(b, (N, N))
    z = _cvec(z, (N, N))
    r = np.empty_like(z)
    lib().or_residual_ld(N, 1.0 / (N + 1), _c(lam), _ptr(b), _ptr(z), _ptr(r))
    return r


def allatonce_residual_ld(N, n, tau, alpha, u, fhat):
    """(||r||_2, r) of eq. (1) with the alpha-circulant B, evaluated in long double and
    rounded to double at the end (a reference below the FP64 rounding of the formula)."""
    u = _rvec(u, (n, N, N))
    fhat = _rvec(fhat, (n, N, N))
    r = np.empty_like(u)
    rn = lib().or_allatonce_residual_ld(N, n, float(tau), float(alpha), _ptr(u), _ptr(fhat), _ptr(r))
    return rn, r


def sequential_backward_euler(N, n, tau, f, u0, kappa=1.0):
    """The system ParaDIAG-II converges to: eq. (1) with alpha = 0, i.e. backward Euler
    stepped in sequence, (I / tau + kappa A) u_k = f_k + u_{k-1} / tau, u_0 the initial
    value, A the five-point Laplacian with h = 1/(N+1) (eq. (1), Sec. 1).  Each step is a
    sparse LU solve (SuperLU through scipy)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    f = _rvec(f, (n, N, N))
    u0 = _rvec(u0, (N, N))
    h = 1.0 / (N + 1)
    T = sp.diags([-np.ones(N - 1), 2.0 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    I = sp.identity(N)
    A = (sp.kron(I, T) + sp.kron(T, I)) / (h * h)
    lu = spl.splu((sp.identity(N * N) / tau + kappa * A).tocsc())
    u = np.empty_like(f)
    prev = u0.ravel()
    for k in range(n):
        prev = lu.solve(f[k].ravel() + prev / tau)
        u[k] = prev.reshape(N, N)
    return u


def set_threads(k):
    """Sets the number of OpenMP threads of the batched oracle routines."""
    lib().or_set_threads(int(k))


def max_threads():
    return int(lib().or_max_threads())
