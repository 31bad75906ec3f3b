"""The C-ABI library builds, loads and exports every entry point of include/paradiag.h;
host-only entry points behave (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import core
from paper_2203_11154_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "paradiag.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = [m for m in re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)
             if m.startswith(("pd_", "paradiag_", "mg_", "shifted_"))]
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    L = C.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert sorted(api.EXPORTS) == names


def test_config_defaults():
    c = api.config()
    assert (c.cycle_gamma, c.nu1, c.nu2, c.coarsest_n, c.maxit) == (1, 1, 1, 3, 100)
    assert c.tol == 1e-10 and c.omega_mode == 1 and c.precision == 0 and c.smoother == 0
    assert c.kappa == 1.0 and c.outer_maxit == 0 and c.max_refine == 12 and c.inner_maxit == 2


def test_shifts_alpha_circulant_is_the_same_closed_form():
    for n, tau, alpha in [(16, 1 / 16, 1e-2), (7, 0.3, 0.5)]:
        sh, V, Vi = api.pd_shifts_alpha_circulant(n, tau, alpha)
        _, sh2, V2, Vi2, _ = api.pd_alpha_circulant(n, tau, alpha)
        assert np.array_equal(sh, sh2) and np.array_equal(V, V2) and np.array_equal(Vi, Vi2)
    with pytest.raises(api.PDError):
        api.pd_shifts_alpha_circulant(4, 0.1, 0.0)


def test_alpha_circulant_matches_oracle():
    for n, tau, alpha in [(16, 1 / 16, 1e-2), (64, 1 / 64, 1e-3), (5, 0.3, 0.5)]:
        B, sh, V, Vi, c0 = api.pd_alpha_circulant(n, tau, alpha)
        lam, Vo, Vio = core.alpha_circulant(n, tau, alpha)
        assert np.allclose(sh, lam, rtol=1e-14, atol=1e-12)
        assert np.allclose(V, Vo, rtol=1e-13, atol=1e-13)
        assert np.allclose(Vi, Vio, rtol=1e-13, atol=1e-16)
        Cm = np.eye(n, k=-1)
        Cm[0, n - 1] = alpha
        assert np.array_equal(B, (np.eye(n) - Cm) / tau)
        assert c0[0] == 1 / tau and not np.any(c0[1:])


def test_setup_rejects_bad_arguments_before_touching_the_gpu():
    L = api.lib()
    h = C.c_void_p()
    sh = np.zeros(8)
    cfg = api.config()
    p = sh.ctypes.data_as(C.c_void_p)
    # N not 2^k - 1, wrong h, n out of range, missing shifts, bad cycle options
    assert L.paradiag_setup(C.byref(h), 10, 1 / 11, 4, p, None, None, None, None, None, C.byref(cfg), None) == 1
    assert L.paradiag_setup(C.byref(h), 7, 0.1, 4, p, None, None, None, None, None, C.byref(cfg), None) == 1
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 0, p, None, None, None, None, None, C.byref(cfg), None) == 1
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 4, None, None, None, None, None, None, C.byref(cfg), None) == 1
    bad = api.config(cycle_gamma=3)
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 4, p, None, None, None, None, None, C.byref(bad), None) == 1
    bad = api.config(coarsest_n=5)
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 4, p, None, None, None, None, None, C.byref(bad), None) == 1
    bad = api.config(precision=1)  # B for the refinement of eq. (1) needs V as well
    Bm = np.eye(4)
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 4, p, None, None, Bm.ctypes.data_as(C.c_void_p), None,
                            None, C.byref(bad), None) == 1
    bad = api.config(cuda_graphs=2)
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 4, p, None, None, None, None, None, C.byref(bad), None) == 1
    bad = api.config(outer_maxit=3)  # FP64 corrections need B and V
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 4, p, None, None, None, None, None, C.byref(bad), None) == 1
    bad = api.config(outer_maxit=-1)
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 4, p, None, None, None, None, None, C.byref(bad), None) == 1
    nan = np.array([np.nan] * 8)
    assert L.paradiag_setup(C.byref(h), 7, 1 / 8, 4, nan.ctypes.data_as(C.c_void_p), None, None, None,
                            None, None, C.byref(cfg), None) == 1
    assert h.value is None


def test_batch_setup_rejects_bad_arguments_before_touching_the_gpu():
    L = api.lib()
    h = C.c_void_p()
    sh = np.array([1.0, 0.5, 2.0, -0.5])
    Ns = (C.c_int * 2)(7, 8)
    ns = (C.c_int * 2)(2, 2)
    sp = (C.c_void_p * 2)(sh.ctypes.data, sh.ctypes.data)
    cfg = api.config()
    args = (C.cast(ns, C.c_void_p), C.cast(sp, C.c_void_p), C.byref(cfg), None)
    assert L.pd_batch_setup(C.byref(h), 2, C.cast(Ns, C.c_void_p), *args) == 1  # N = 8
    assert L.pd_batch_setup(C.byref(h), 0, C.cast(Ns, C.c_void_p), *args) == 1
    assert L.pd_batch_setup(C.byref(h), 65, C.cast(Ns, C.c_void_p), *args) == 1
    bad = api.config(omega_mode=2)
    Ns[1] = 15
    assert L.pd_batch_setup(C.byref(h), 2, C.cast(Ns, C.c_void_p), C.cast(ns, C.c_void_p),
                            C.cast(sp, C.c_void_p), C.byref(bad), None) == 1
    assert h.value is None
    assert L.pd_batch_destroy(None) == 1
    assert L.pd_batch_last_error(None) == b""


def test_status_strings():
    L = api.lib()
    for code in range(8):
        assert L.pd_status_str(code)
    assert L.pd_status_str(99) == b"unknown status"


def _qbvm(n, beta):
    """B of eq. (10), (n+1) x (n+1), tau = 1/n."""
    B = np.eye(n + 1) - np.eye(n + 1, k=-1)
    B[0, n] = 1.0 / beta
    return B * n


@pytest.mark.parametrize("which,n", [("ex1", 16), ("ex1", 128), ("ex1", 256), ("ex2", 15),
                                     ("ex2", 127), ("alpha", 64), ("random", 40)])
def test_diagonalize_reconstructs_B(which, n):
    """pd_diagonalize (the set-up diagonalisation of Sec. 1) on Example 1's BVM B (eq. (9)),
    Example 2's quasi-BVM B (eq. (10)), the alpha-circulant B and a random matrix: V D V^{-1}
    rebuilds B and V V^{-1} = I to cond(V) times a few ulps, the eigenvalues are numpy's
    (LAPACK), and Example 1's bound |lam| < n + sqrt(n)/sqrt(2) holds."""
    from oracle import lfa
    if which == "ex1":
        B = lfa.ex1_bvm_matrix(n)
    elif which == "ex2":
        B = _qbvm(n, 0.01)
    elif which == "alpha":
        B = api.pd_alpha_circulant(n, 1.0 / n, 1e-3)[0]
    else:
        B = np.random.default_rng(7).standard_normal((n, n))
    m = B.shape[0]
    lam, V, Vi = api.pd_diagonalize(B)
    condV = np.linalg.cond(V)
    eps = np.finfo(float).eps
    nb = np.linalg.norm(B, 2)
    rec = V @ np.diag(lam) @ Vi
    assert np.linalg.norm(rec - B, 2) <= 50 * m * eps * condV * nb
    assert np.linalg.norm(V @ Vi - np.eye(m), 2) <= 50 * m * eps * condV
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0, rtol=1e-14)
    ref = np.linalg.eigvals(B)
    # match every computed eigenvalue to the nearest LAPACK one (distinct eigenvalues)
    d = np.abs(lam[:, None] - ref[None, :])
    assert np.array_equal(np.sort(np.argmin(d, axis=1)), np.arange(m))
    assert np.max(np.min(d, axis=1)) <= 1e-9 * np.max(np.abs(ref))
    if which == "ex1":
        assert np.max(np.abs(lam)) < n + np.sqrt(n) / np.sqrt(2)


def test_diagonalize_rejects_bad_input():
    with pytest.raises(api.PDError):
        api.pd_diagonalize(np.array([[1.0, np.nan], [0.0, 2.0]]))
    # a Jordan block is not diagonalisable: V comes out singular in FP64
    with pytest.raises(api.PDError):
        api.pd_diagonalize(np.array([[1.0, 1.0], [0.0, 1.0]]))
