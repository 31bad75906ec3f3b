"""Thin ctypes binding of libparadiag.so (include/paradiag.h), same names as the C ABI.

Only argument marshalling happens here: torch CUDA tensors become device pointers,
numpy arrays become host pointers, status codes become exceptions.  Every step of a
solve runs in the library's kernels.  The library must have been built (see
`build.build()`); if it is missing or cannot be loaded this module raises instead of
falling back to anything else.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

PD_STAT_RELRES_ALLATONCE = 0
PD_STAT_REFINE_STEPS = 1
PD_STAT_IMAG_MAX = 2
PD_STAT_CYCLES_TOTAL = 3
PD_STAT_CYCLES_MAX = 4
PD_STAT_RELRES_SHIFT_MAX = 5
PD_STATS_LEN = 8

KERNEL_CLASSES = ["smooth0", "restrict0", "prolong0", "smooth_c", "restrict_c", "prolong_c",
                  "coarse", "converge", "forward", "inverse", "residual", "other",
                  "smooth_restrict0", "prolong_smooth0", "smooth_restrict_c", "prolong_smooth_c"]

STATUS = {0: "PD_OK", 1: "PD_ERR_ARG", 2: "PD_ERR_CUDA", 3: "PD_ERR_NOMEM", 4: "PD_ERR_NOCONV",
          5: "PD_ERR_NAN", 6: "PD_ERR_SING", 7: "PD_ERR_STATE"}

EXPORTS = ["pd_config_default", "pd_alpha_circulant", "pd_shifts_alpha_circulant", "pd_diagonalize",
           "paradiag_setup",
           "pd_adjoint_setup",
           "pd_num_levels",
           "pd_get_omega", "mg_vcycle", "shifted_solve_batched", "paradiag_solve",
           "paradiag_solve_host", "pd_smooth", "pd_residual_restrict", "pd_prolong_add",
           "pd_coarse_solve", "pd_transform_forward", "pd_transform_inverse",
           "pd_allatonce_residual", "pd_allatonce_residual_static", "pd_laplacian_dot",
           "pd_initial_value_gradient",
           "pd_profile_enable", "pd_profile_read", "pd_get_history", "pd_synchronize", "pd_launch_count", "pd_batch_launch_count", "pd_fused_choice", "paradiag_destroy",
           "pd_status_str", "pd_last_error", "shifted_solve_refined", "pd_allatonce_residual32", "pd_shifted_residual32",
           "paradiag_solve_host_batch", "pd_batch_setup",
           "pd_batch_solve", "pd_batch_destroy", "pd_batch_last_error", "pd_batch_info"]


class PDError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        self.status = STATUS.get(code, str(code))
        super().__init__("%s: %s%s" % (where, self.status, (" (%s)" % detail) if detail else ""))


class pd_config(C.Structure):
    _fields_ = [("cycle_gamma", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("coarsest_n", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("omega_mode", C.c_int), ("precision", C.c_int), ("smoother", C.c_int),
                ("inner_tol", C.c_double), ("max_refine", C.c_int), ("imag_check", C.c_int),
                ("inner_maxit", C.c_int), ("stall_ratio", C.c_double), ("fused", C.c_int),
                ("tensor_transforms", C.c_int), ("fused_variant", C.c_int),
                ("kappa", C.c_double), ("outer_maxit", C.c_int), ("cuda_graphs", C.c_int),
                ("fx_residual", C.c_int), ("fft_transforms", C.c_int)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double


def lib(path=None):
    """Loads libparadiag.so (building it first if it is out of date)."""
    global _lib
    if _lib is None:
        if path is None:
            path = _build.LIB
            if not _build.up_to_date():
                _build.build()
        if not os.path.exists(path):
            raise ImportError("libparadiag.so not found at %s" % path)
        L = C.CDLL(path)
        sig = {
            "pd_config_default": (None, [C.POINTER(pd_config)]),
            "pd_alpha_circulant": (_I, [_I, _D, _D, _P, _P, _P, _P, _P]),
            "pd_shifts_alpha_circulant": (_I, [_I, _D, _D, _P, _P, _P]),
            "pd_diagonalize": (_I, [_I, _P, _P, _P, _P]),
            "paradiag_setup": (_I, [C.POINTER(_P), _I, _D, _I, _P, _P, _P, _P, _P, _P,
                                    C.POINTER(pd_config), _P]),
            "pd_adjoint_setup": (_I, [_P, C.POINTER(_P)]),
            "pd_num_levels": (_I, [_P]),
            "pd_get_omega": (_I, [_P, _P]),
            "mg_vcycle": (_I, [_P, _I, _P, _P]),
            "shifted_solve_batched": (_I, [_P, _P, _P, _P, _P]),
            "paradiag_solve": (_I, [_P, _P, _P, _P, _P, _P, _P]),
            "paradiag_solve_host": (_I, [_P, _P, _P, _P, _P, _P, _P]),
            "pd_smooth": (_I, [_P, _I, _P, _P, _P]),
            "pd_residual_restrict": (_I, [_P, _I, _P, _P, _P]),
            "pd_prolong_add": (_I, [_P, _I, _P, _P]),
            "pd_coarse_solve": (_I, [_P, _P, _P]),
            "pd_transform_forward": (_I, [_P, _P, _P, _P]),
            "pd_transform_inverse": (_I, [_P, _P, _P, _I]),
            "pd_allatonce_residual": (_I, [_P, _P, _P, _P, _P, _P]),
            "pd_allatonce_residual_static": (_I, [_I, _I, _D, _D, _P, _P, _P, _P, _P, _P]),
            "pd_laplacian_dot": (_I, [_P, _P, _P, _P]),
            "pd_initial_value_gradient": (_I, [_P, _P, _P]),
            "pd_profile_enable": (_I, [_P, _I]),
            "pd_profile_read": (_I, [_P, _I, _P, _P, _P]),
            "pd_get_history": (_I, [_P, _I, _P, _P, _I, _P, _P]),
            "pd_synchronize": (_I, [_P]),
            "pd_launch_count": (C.c_longlong, [_P]),
            "pd_batch_launch_count": (C.c_longlong, [_P]),
            "pd_fused_choice": (_I, [_P, _I, _P, _P]),
            "paradiag_destroy": (_I, [_P]),
            "pd_status_str": (C.c_char_p, [_I]),
            "pd_last_error": (C.c_char_p, [_P]),
            "shifted_solve_refined": (_I, [_P, _P, _P, _P, _P]),
            "pd_allatonce_residual32": (_I, [_P, _P, _P, _P, _P, _P]),
            "pd_shifted_residual32": (_I, [_P, _P, _P, _P, _P]),
            "paradiag_solve_host_batch": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
            "pd_batch_setup": (_I, [C.POINTER(_P), _I, _P, _P, _P, C.POINTER(pd_config), _P]),
            "pd_batch_solve": (_I, [_P, _P, _P, _P, _P]),
            "pd_batch_destroy": (_I, [_P]),
            "pd_batch_last_error": (C.c_char_p, [_P]),
            "pd_batch_info": (_I, [_P, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def config(**kw):
    """pd_config with the library defaults, then the given fields."""
    c = pd_config()
    lib().pd_config_default(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError("pd_config has no field %r" % k)
        setattr(c, k, v)
    return c


def _dptr(t, dtype=None, numel=None):
    """Device pointer of a contiguous CUDA tensor (checked)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError("expected %s, got %s" % (dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d elements, got %d" % (numel, t.numel()))
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(code, where, ctx=None):
    if code != 0:
        detail = ""
        if ctx is not None:
            detail = (lib().pd_last_error(ctx) or b"").decode(errors="replace")
        raise PDError(code, where, detail)


def pd_alpha_circulant(n, tau, alpha):
    """(B [n][n], shifts [n] complex, V, Vinv [n][n] complex, u0_coef [n])."""
    B = np.zeros((n, n))
    sh = np.zeros(2 * n)
    V = np.zeros(2 * n * n)
    Vi = np.zeros(2 * n * n)
    c0 = np.zeros(n)
    _check(lib().pd_alpha_circulant(n, float(tau), float(alpha), _hptr(B), _hptr(sh), _hptr(V),
                                    _hptr(Vi), _hptr(c0)), "pd_alpha_circulant")
    return B, sh.view(np.complex128), V.view(np.complex128).reshape(n, n), \
        Vi.view(np.complex128).reshape(n, n), c0


def pd_shifts_alpha_circulant(n, tau, alpha):
    """(shifts [n] complex, V, Vinv [n][n] complex)."""
    sh = np.zeros(2 * n)
    V = np.zeros(2 * n * n)
    Vi = np.zeros(2 * n * n)
    _check(lib().pd_shifts_alpha_circulant(n, float(tau), float(alpha), _hptr(sh), _hptr(V), _hptr(Vi)),
           "pd_shifts_alpha_circulant")
    return sh.view(np.complex128), V.view(np.complex128).reshape(n, n), Vi.view(np.complex128).reshape(n, n)


class Context:
    """A paradiag context (one GPU, the caller's current torch stream)."""

    def __init__(self, N, n, shifts, V=None, Vinv=None, B=None, u0_coef=None, omega=None,
                 cfg=None, stream=None):
        import torch
        self.N, self.n = int(N), int(n)
        self.cfg = cfg if cfg is not None else config()
        if shifts is None:
            sh = None
            self._keep = []
            args = [None]
        else:
            sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.complex128).reshape(n))
            self._keep = [sh]
            args = [_hptr(sh.view(np.float64))]
        for a in (V, Vinv):
            if a is None:
                args.append(None)
            else:
                a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128).reshape(n, n))
                self._keep.append(a)
                args.append(_hptr(a.view(np.float64)))
        for a in (B, u0_coef, omega):
            if a is None:
                args.append(None)
            else:
                a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
                self._keep.append(a)
                args.append(_hptr(a))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = C.c_void_p()
        _check(lib().paradiag_setup(C.byref(h), self.N, 1.0 / (self.N + 1), self.n, *args,
                                    C.byref(self.cfg), C.c_void_p(stream)), "paradiag_setup")
        self.h = h
        self.levels = lib().pd_num_levels(h)
        self.Ns = [self.N]
        while len(self.Ns) < self.levels:
            self.Ns.append((self.Ns[-1] - 1) // 2)
        self.ctype = torch.complex128 if self.cfg.precision == 0 else torch.complex64

    # -- helpers -------------------------------------------------------------------
    def omega(self):
        out = np.zeros((self.n, self.levels))
        _check(lib().pd_get_omega(self.h, _hptr(out)), "pd_get_omega", self.h)
        return out

    def _grid(self, t, level=0, dtype=None):
        N = self.Ns[level]
        return _dptr(t, dtype or self.ctype, self.n * N * N)

    def synchronize(self):
        _check(lib().pd_synchronize(self.h), "pd_synchronize", self.h)

    def adjoint(self):
        """Context of the transposed step (pd_adjoint_setup)."""
        a = Context.__new__(Context)
        h = C.c_void_p()
        _check(lib().pd_adjoint_setup(self.h, C.byref(h)), "pd_adjoint_setup", self.h)
        a.h = h
        a.N, a.n, a.cfg, a.stream, a._keep = self.N, self.n, self.cfg, self.stream, []
        a.levels, a.Ns, a.ctype = self.levels, list(self.Ns), self.ctype
        return a

    def history(self, cap=None, cap_outer=64):
        """(cycle_hist: list of n arrays, the per-shift relative residuals before the first
        and after each cycle of the last multigrid solve; outer: array of the relative
        residuals of eq. (1) after each step of the last paradiag_solve)."""
        if cap is None:
            cap = max(self.cfg.maxit, self.cfg.inner_maxit) + 1
        ln = np.zeros(self.n, np.int32)
        h = np.zeros((self.n, cap))
        lo = C.c_int()
        ho = np.zeros(cap_outer)
        _check(lib().pd_get_history(self.h, cap, _hptr(ln), _hptr(h), cap_outer, C.byref(lo), _hptr(ho)),
               "pd_get_history", self.h)
        return [h[j, :ln[j]].copy() for j in range(self.n)], ho[:lo.value].copy()

    def history_jsonl(self):
        """The convergence history of the last solve as JSON lines: one line per shift
        ({"shift": j, "relres": [...]}), then one for eq. (1) ({"allatonce_relres": [...]})."""
        import json
        cyc, outer = self.history()
        lines = [json.dumps({"shift": j, "relres": [float(x) for x in h]}) for j, h in enumerate(cyc)]
        lines.append(json.dumps({"allatonce_relres": [float(x) for x in outer]}))
        return "\n".join(lines)

    def launch_count(self):
        return int(lib().pd_launch_count(self.h))

    def fused_choices(self):
        """Per multigrid level: (variant, rows per segment) of the fused smoothing kernels
        the autotuner chose (1 TMA tiles, 2 warp streams, 0 none)."""
        out = []
        for l in range(lib().pd_num_levels(self.h)):
            v, sg = C.c_int(), C.c_int()
            _check(lib().pd_fused_choice(self.h, l, C.byref(v), C.byref(sg)), "pd_fused_choice", self.h)
            out.append((v.value, sg.value))
        return out

    def profile_enable(self, on=True):
        _check(lib().pd_profile_enable(self.h, int(bool(on))), "pd_profile_enable", self.h)

    def profile_read(self):
        """{class: (total_ms, launches, algorithmic_bytes)} since profile_enable."""
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            ms = C.c_double()
            nl = C.c_longlong()
            by = C.c_double()
            _check(lib().pd_profile_read(self.h, k, C.byref(ms), C.byref(nl), C.byref(by)),
                   "pd_profile_read", self.h)
            out[name] = (ms.value, nl.value, by.value)
        return out

    def destroy(self):
        if getattr(self, "h", None):
            lib().paradiag_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # -- the C ABI -----------------------------------------------------------------
    def mg_vcycle(self, level, z, b):
        _check(lib().mg_vcycle(self.h, level, self._grid(z, level), self._grid(b, level)),
               "mg_vcycle", self.h)

    def shifted_solve_batched(self, z, b, raise_on_noconv=True):
        it = np.zeros(self.n, np.int32)
        rr = np.zeros(self.n)
        code = lib().shifted_solve_batched(self.h, self._grid(z), self._grid(b), _hptr(it), _hptr(rr))
        if code != 0 and not (code == 4 and not raise_on_noconv):
            _check(code, "shifted_solve_batched", self.h)
        return it, rr

    def shifted_solve_refined(self, z, b, raise_on_noconv=True):
        """z, b: complex128 [n][N][N] device tensors (FP64 answer for either precision)."""
        import torch
        it = np.zeros(self.n, np.int32)
        rr = np.zeros(self.n)
        m = self.n * self.N * self.N
        code = lib().shifted_solve_refined(self.h, _dptr(z, torch.complex128, m),
                                           _dptr(b, torch.complex128, m), _hptr(it), _hptr(rr))
        if code != 0 and not (code == 4 and not raise_on_noconv):
            _check(code, "shifted_solve_refined", self.h)
        return it, rr

    def _solve_out(self, code, it, rr, stats, where, raise_on_noconv):
        if code != 0 and not (code == 4 and not raise_on_noconv):
            _check(code, where, self.h)
        return dict(iters=it, relres=rr, relres_allatonce=stats[PD_STAT_RELRES_ALLATONCE],
                    refine_steps=int(stats[PD_STAT_REFINE_STEPS]), imag_max=stats[PD_STAT_IMAG_MAX],
                    cycles_total=int(stats[PD_STAT_CYCLES_TOTAL]),
                    cycles_max=int(stats[PD_STAT_CYCLES_MAX]),
                    relres_shift_max=stats[PD_STAT_RELRES_SHIFT_MAX], status=STATUS.get(code))

    def paradiag_solve(self, u, f, u0=None, raise_on_noconv=True):
        import torch
        it = np.zeros(self.n, np.int32)
        rr = np.zeros(self.n)
        stats = np.zeros(PD_STATS_LEN)
        m = self.n * self.N * self.N
        code = lib().paradiag_solve(self.h, _dptr(u, torch.float64, m), _dptr(f, torch.float64, m),
                                    _dptr(u0, torch.float64, self.N * self.N), _hptr(it),
                                    _hptr(rr), _hptr(stats))
        return self._solve_out(code, it, rr, stats, "paradiag_solve", raise_on_noconv)

    @staticmethod
    def _host_ptr(a, numel):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous() or a.numel() != numel:
                raise ValueError("expected a contiguous host tensor of %d elements" % numel)
            return C.c_void_p(a.data_ptr())
        a = np.asarray(a)
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != numel:
            raise ValueError("expected a contiguous float64 array of %d elements" % numel)
        return _hptr(a)

    def paradiag_solve_host_batch(self, us, fs, u0s=None, raise_on_noconv=True):
        """count steps with host buffers, copies pipelined with the solves; us, fs (and u0s)
        are lists of contiguous float64 host tensors or arrays.  Returns a list of result
        dicts (as paradiag_solve)."""
        k = len(fs)
        if len(us) != k or (u0s is not None and len(u0s) != k):
            raise ValueError("one u (and u0) per f")
        m = self.n * self.N * self.N
        up = (C.c_void_p * k)(*[self._host_ptr(a, m).value for a in us])
        fp = (C.c_void_p * k)(*[self._host_ptr(a, m).value for a in fs])
        u0p = None
        if u0s is not None:
            u0p = (C.c_void_p * k)(*[(self._host_ptr(a, self.N * self.N).value if a is not None else None)
                                     for a in u0s])
        it = np.zeros(k * self.n, np.int32)
        rr = np.zeros(k * self.n)
        stats = np.zeros(k * PD_STATS_LEN)
        code = lib().paradiag_solve_host_batch(self.h, k, C.cast(up, C.c_void_p), C.cast(fp, C.c_void_p),
                                               C.cast(u0p, C.c_void_p) if u0p is not None else None,
                                               _hptr(it), _hptr(rr), _hptr(stats))
        if code != 0 and not (code == 4 and not raise_on_noconv):
            _check(code, "paradiag_solve_host_batch", self.h)
        return [self._solve_out(0, it[j * self.n:(j + 1) * self.n], rr[j * self.n:(j + 1) * self.n],
                                stats[j * PD_STATS_LEN:(j + 1) * PD_STATS_LEN],
                                "paradiag_solve_host_batch", False) for j in range(k)]

    def paradiag_solve_host(self, u, f, u0=None, raise_on_noconv=True):
        """u, f, u0: contiguous float64 host tensors or numpy arrays (pinned is fastest)."""
        hp = self._host_ptr
        it = np.zeros(self.n, np.int32)
        rr = np.zeros(self.n)
        stats = np.zeros(PD_STATS_LEN)
        m = self.n * self.N * self.N
        code = lib().paradiag_solve_host(self.h, hp(u, m), hp(f, m), hp(u0, self.N * self.N),
                                         _hptr(it), _hptr(rr), _hptr(stats))
        return self._solve_out(code, it, rr, stats, "paradiag_solve_host", raise_on_noconv)

    def pd_smooth(self, level, z_out, z_in, b):
        _check(lib().pd_smooth(self.h, level, self._grid(z_out, level), self._grid(z_in, level),
                               self._grid(b, level)), "pd_smooth", self.h)

    def pd_residual_restrict(self, level, bc, z, b):
        _check(lib().pd_residual_restrict(self.h, level, self._grid(bc, level + 1),
                                          self._grid(z, level), self._grid(b, level)),
               "pd_residual_restrict", self.h)

    def pd_prolong_add(self, level, z, ec):
        _check(lib().pd_prolong_add(self.h, level, self._grid(z, level), self._grid(ec, level + 1)),
               "pd_prolong_add", self.h)

    def pd_coarse_solve(self, z, b):
        L = self.levels - 1
        _check(lib().pd_coarse_solve(self.h, self._grid(z, L), self._grid(b, L)),
               "pd_coarse_solve", self.h)

    def pd_transform_forward(self, g, f, u0=None):
        import torch
        m = self.n * self.N * self.N
        _check(lib().pd_transform_forward(self.h, self._grid(g), _dptr(f, torch.float64, m),
                                          _dptr(u0, torch.float64, self.N * self.N)),
               "pd_transform_forward", self.h)

    def pd_transform_inverse(self, u, z, accumulate=False):
        import torch
        m = self.n * self.N * self.N
        _check(lib().pd_transform_inverse(self.h, _dptr(u, torch.float64, m), self._grid(z),
                                          int(bool(accumulate))), "pd_transform_inverse", self.h)

    def pd_laplacian_dot(self, w, u):
        """sum_k <w_k, A u_k> (FP64)."""
        import torch
        m = self.n * self.N * self.N
        out = C.c_double()
        _check(lib().pd_laplacian_dot(self.h, _dptr(w, torch.float64, m), _dptr(u, torch.float64, m),
                                      C.byref(out)), "pd_laplacian_dot", self.h)
        return out.value

    def pd_initial_value_gradient(self, w, gu0):
        import torch
        m = self.n * self.N * self.N
        _check(lib().pd_initial_value_gradient(self.h, _dptr(w, torch.float64, m),
                                               _dptr(gu0, torch.float64, self.N * self.N)),
               "pd_initial_value_gradient", self.h)

    def pd_allatonce_residual(self, r, u, f, u0=None):
        import torch
        m = self.n * self.N * self.N
        norms = np.zeros(2)
        _check(lib().pd_allatonce_residual(self.h, _dptr(r, torch.float64, m),
                                           _dptr(u, torch.float64, m), _dptr(f, torch.float64, m),
                                           _dptr(u0, torch.float64, self.N * self.N), _hptr(norms)),
               "pd_allatonce_residual", self.h)
        return norms[0], norms[1]

    def pd_allatonce_residual32(self, r32, u, f, u0=None):
        """r32: float32 [n][N][N] device tensor; returns (||r||, ||fhat||)."""
        import torch
        m = self.n * self.N * self.N
        norms = np.zeros(2)
        _check(lib().pd_allatonce_residual32(self.h, _dptr(r32, torch.float32, m),
                                             _dptr(u, torch.float64, m), _dptr(f, torch.float64, m),
                                             _dptr(u0, torch.float64, self.N * self.N), _hptr(norms)),
               "pd_allatonce_residual32", self.h)
        return norms[0], norms[1]

    def pd_shifted_residual32(self, r32, z, b):
        """r32: complex64 [n][N][N]; z, b: complex128 [n][N][N] device tensors.  Returns the
        per-shift ||r_j||."""
        import torch
        m = self.n * self.N * self.N
        norms = np.zeros(self.n)
        _check(lib().pd_shifted_residual32(self.h, _dptr(r32, torch.complex64, m),
                                           _dptr(z, torch.complex128, m), _dptr(b, torch.complex128, m),
                                           _hptr(norms)), "pd_shifted_residual32", self.h)
        return norms


def paradiag_setup(N, n, shifts, V=None, Vinv=None, B=None, u0_coef=None, omega=None, cfg=None,
                   stream=None):
    return Context(N, n, shifts, V, Vinv, B, u0_coef, omega, cfg, stream)


def alpha_circulant_context(N, n, tau, alpha, **cfg_fields):
    """Context for the backward-Euler alpha-circulant ParaDIAG step on an N x N grid."""
    B, sh, V, Vi, c0 = pd_alpha_circulant(n, tau, alpha)
    return Context(N, n, sh, V, Vi, B, c0, None, config(**cfg_fields))


def paradiag2_context(N, n, tau, alpha, **cfg_fields):
    """ParaDIAG-II for sequential backward Euler: the residual of eq. (1) uses the lower-
    bidiagonal B_0 = (1/tau)(I - C_0) (no corner), the solves use the shifts and V of the
    alpha-circulant B_alpha, so each correction step contracts the error by about
    alpha / (1 - alpha).  Precision 1 refines with it by construction; precision 0 needs
    outer_maxit > 0 (set to 20 here unless given)."""
    B, sh, V, Vi, c0 = pd_alpha_circulant(n, tau, alpha)
    B = B.copy()
    if n > 1:
        B[0, n - 1] = 0.0
    cfg_fields.setdefault("outer_maxit", 20 if cfg_fields.get("precision", 0) == 0 else 0)
    return Context(N, n, sh, V, Vi, B, c0, None, config(**cfg_fields))


def pd_diagonalize(B):
    """(shifts [n] complex, V, Vinv [n][n] complex) of the real n x n B = V D V^{-1},
    computed by the library on the host."""
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float64))
    n = B.shape[0]
    if B.shape != (n, n):
        raise ValueError("B must be square")
    sh = np.zeros(2 * n)
    V = np.zeros(2 * n * n)
    Vi = np.zeros(2 * n * n)
    _check(lib().pd_diagonalize(n, _hptr(B), _hptr(sh), _hptr(V), _hptr(Vi)), "pd_diagonalize")
    return sh.view(np.complex128), V.view(np.complex128).reshape(n, n), Vi.view(np.complex128).reshape(n, n)


def dense_B_context(B, N, u0_coef=None, **cfg_fields):
    """Context for eq. (1) with a general diagonalisable time matrix B (n x n real), e.g.
    the boundary-value-method B of Example 1 (eq. (9)) or the quasi-BVM B of Example 2
    (eq. (10)).  Only B is passed: paradiag_setup diagonalises it (B = V D V^{-1})."""
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float64))
    n = B.shape[0]
    return Context(N, n, None, None, None, B, u0_coef, None, config(**cfg_fields))


class Batch:
    """pd_batch: independent shifted-system problems of uneven sizes solved together
    (instance i: N_i x N_i grid, shifts[i] of length n_i)."""

    def __init__(self, Ns, shifts, cfg=None, stream=None):
        import torch
        self.Ns = [int(N) for N in Ns]
        self.shifts = [np.ascontiguousarray(np.asarray(s, dtype=np.complex128).ravel()) for s in shifts]
        self.ns = [s.size for s in self.shifts]
        k = len(self.Ns)
        if len(self.shifts) != k:
            raise ValueError("one shift array per instance")
        self.cfg = cfg if cfg is not None else config()
        Narr = (C.c_int * k)(*self.Ns)
        narr = (C.c_int * k)(*self.ns)
        sarr = (C.c_void_p * k)(*[s.ctypes.data for s in self.shifts])
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        code = lib().pd_batch_setup(C.byref(h), k, C.cast(Narr, C.c_void_p), C.cast(narr, C.c_void_p),
                                    C.cast(sarr, C.c_void_p), C.byref(self.cfg), C.c_void_p(stream))
        if code != 0:
            raise PDError(code, "pd_batch_setup", "")
        self.h = h

    def solve(self, zs, bs, raise_on_noconv=True):
        """zs, bs: lists of complex128 [n_i][N_i][N_i] device tensors.  Returns per-instance
        (iters, relres) lists."""
        import torch
        k = len(self.Ns)
        zp = (C.c_void_p * k)(*[_dptr(z, torch.complex128, n * N * N).value
                                for z, n, N in zip(zs, self.ns, self.Ns)])
        bp = (C.c_void_p * k)(*[_dptr(b, torch.complex128, n * N * N).value
                                for b, n, N in zip(bs, self.ns, self.Ns)])
        tot = sum(self.ns)
        it = np.zeros(tot, np.int32)
        rr = np.zeros(tot)
        code = lib().pd_batch_solve(self.h, C.cast(zp, C.c_void_p), C.cast(bp, C.c_void_p),
                                    _hptr(it), _hptr(rr))
        if code != 0 and not (code == 4 and not raise_on_noconv):
            detail = lib().pd_batch_last_error(self.h).decode(errors="replace")
            raise PDError(code, "pd_batch_solve", detail)
        out, o = [], 0
        for n in self.ns:
            out.append((it[o:o + n].copy(), rr[o:o + n].copy()))
            o += n
        return out

    def info(self):
        """(batched: one launch per level over all instances, launches per cycle, batched
        launches so far)."""
        b = C.c_int()
        lpc = C.c_int()
        tot = C.c_longlong()
        _check(lib().pd_batch_info(self.h, C.byref(b), C.byref(lpc), C.byref(tot)), "pd_batch_info")
        return bool(b.value), lpc.value, tot.value

    def launch_count(self):
        """Every kernel launch of the batch so far (batched multigrid and per instance)."""
        return int(lib().pd_batch_launch_count(self.h))

    def destroy(self):
        if getattr(self, "h", None):
            lib().pd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
