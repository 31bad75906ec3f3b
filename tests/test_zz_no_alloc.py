"""pd_allatonce_residual_static: the residual check that allocates nothing, for callers
that cannot call cudaMalloc (their own memory pool owns the device, or a time-critical
loop cannot take cudaMalloc's synchronisation).  Checked through the C ABI against the
context-based pd_allatonce_residual on two calls in a row, and element by element against
the oracle's residual of eq. (1).  This file is collected last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_2203_11154_gb300 import api, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_static_residual_matches_context_entry_point_twice():
    N, n, tau, alpha = 63, 16, 1.0 / 16, 1e-3
    f, u0 = inputs.paradiag_problem(N, n, seed=7)
    rng = np.random.default_rng(8)
    ctx = api.alpha_circulant_context(N, n, tau, alpha)
    L = api.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    fd = torch.from_numpy(f).cuda()
    u0d = torch.from_numpy(u0).cuda()
    for call in range(2):
        u = torch.from_numpy(rng.standard_normal((n, N, N)) * (call + 1)).cuda()
        r_ref = torch.empty_like(u)
        rn, fn = ctx.pd_allatonce_residual(r_ref, u, fd, u0d)
        r = torch.full_like(u, np.nan)
        norms = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
        code = L.pd_allatonce_residual_static(N, n, tau, alpha, C.c_void_p(u.data_ptr()),
                                              C.c_void_p(fd.data_ptr()), C.c_void_p(u0d.data_ptr()),
                                              C.c_void_p(r.data_ptr()), C.c_void_p(norms.data_ptr()),
                                              stream)
        assert code == 0
        torch.cuda.synchronize()
        nh = norms.cpu().numpy()
        assert abs(nh[0] - rn) <= 1e-12 * rn and abs(nh[1] - fn) <= 1e-12 * fn
        rel = torch.linalg.norm(r - r_ref) / torch.linalg.norm(r_ref)
        assert float(rel) <= 1e-14
        # the oracle's FP64 residual: two FP64 evaluations of the same formula differ by
        # their rounding, 8 eps (|fhat| + |B||u| + |A||u|) per element at most
        uh = u.cpu().numpy()
        fhat = core.assemble_rhs(N, n, tau, f, u0)
        rn_o, fn_o, r_o = core.allatonce_residual(N, n, tau, alpha, uh, fhat, want_r=True)
        h2 = float((N + 1) ** 2)
        au = np.abs(uh)
        nb = np.zeros_like(au)
        nb[:, 1:, :] += au[:, :-1, :]
        nb[:, :-1, :] += au[:, 1:, :]
        nb[:, :, 1:] += au[:, :, :-1]
        nb[:, :, :-1] += au[:, :, 1:]
        wprev = np.ones(n)
        wprev[0] = alpha  # (C_alpha u)_k = u_{k-1}, and alpha u_{n-1} for k = 0
        bu = (au + wprev[:, None, None] * np.roll(au, 1, axis=0)) / tau
        bound = 8 * np.finfo(float).eps * (np.abs(fhat) + bu + h2 * (4 * au + nb))
        assert np.all(np.abs(r.cpu().numpy() - r_o) <= bound)
        assert abs(nh[0] - rn_o) <= 1e-12 * rn_o and abs(nh[1] - fn_o) <= 1e-12 * fn_o


def test_static_residual_rejects_sizes_beyond_its_scratch():
    L = api.lib()
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = C.c_void_p(d.data_ptr())
    assert L.pd_allatonce_residual_static(1, 129, 1.0, 0.5, p, p, None, None, p, None) == 1
    assert L.pd_allatonce_residual_static(0, 4, 1.0, 0.5, p, p, None, None, p, None) == 1
