"""pd_allatonce_residual_static: the residual check that allocates nothing, for callers
that cannot call cudaMalloc (their own memory pool owns the device, or a time-critical
loop cannot take cudaMalloc's synchronisation).  Checked through the C ABI against the
context-based pd_allatonce_residual on two calls in a row.  This file is collected last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def test_static_residual_rejects_sizes_beyond_its_scratch():
    L = api.lib()
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = C.c_void_p(d.data_ptr())
    assert L.pd_allatonce_residual_static(1, 129, 1.0, 0.5, p, p, None, None, p, None) == 1
    assert L.pd_allatonce_residual_static(0, 4, 1.0, 0.5, p, p, None, None, p, None) == 1
