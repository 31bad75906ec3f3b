"""GPU parity of the time transforms, the all-at-once residual and the whole ParaDIAG
step (FP64 and the FP32 + FP64-refinement form) against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core, lfa  # noqa: E402
from paper_2203_11154_gb300 import api, inputs  # noqa: E402


def rel_per_vector(x, ref):
    x = np.asarray(x).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.max(np.linalg.norm(x - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300))


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def gamma_weights(n, alpha):
    """Gamma = diag(alpha^{k/n}): V = Gamma^{-1} Fbar, so Gamma u = Fbar z."""
    return alpha ** (np.arange(n) / n)


def weighted_rel_err(u, ref, alpha):
    """||Gamma (u - ref)|| / ||Gamma ref||: the difference of two FP64 solutions in the norm
    in which (V kron I) is an isometry up to sqrt(n), so that the alpha^{-(k-1)/n}
    amplification of the late time steps by V does not enter."""
    n = ref.shape[0]
    g = gamma_weights(n, alpha)[:, None, None]
    return np.linalg.norm(g * (u - ref)) / np.linalg.norm(g * ref)


def residual_error_bound(N, n, alpha, rr1, rr2, fnorm):
    """||u1 - u2|| <= ||A^{-1}|| (||r1|| + ||r2||) with ||A^{-1}|| <= cond(V) max_j
    ||(lam_j + A)^{-1}|| <= alpha^{-(n-1)/n} / mu_min, mu_min = (8/h^2) sin^2(pi h / 2) the
    smallest eigenvalue of A (Re lam_j > 0 for the alpha-circulant shifts)."""
    h = 1.0 / (N + 1)
    mu = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    return alpha ** (-(n - 1) / n) / mu * (rr1 + rr2) * fnorm


def residual_rounding(N, n, tau, alpha, u, fhat):
    """8 eps || |fhat| + |B| |u| + |A| |u| ||: a bound on the difference between two FP64
    evaluations of ||fhat - (B kron I + I kron A) u|| in different operation orders, which
    dominates once the residual reaches the FP64 floor."""
    h = 1.0 / (N + 1)
    a = np.abs(u)
    nb = np.zeros_like(a)
    nb[:, 1:, :] += a[:, :-1, :]
    nb[:, :-1, :] += a[:, 1:, :]
    nb[:, :, 1:] += a[:, :, :-1]
    nb[:, :, :-1] += a[:, :, 1:]
    prev = np.roll(a, 1, axis=0)
    prev[0] *= alpha
    t = np.abs(fhat) + (a + prev) / tau + (4 * a + nb) / h ** 2
    return 8 * np.finfo(float).eps * np.linalg.norm(t)


def oracle_paradiag(N, n, tau, alpha, f, u0, omega_mode="lfa", tol=1e-10):
    lam, V, Vinv = core.alpha_circulant(n, tau, alpha)
    om = lfa.omega_table(lam, N, mode=omega_mode)
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    u, im, iters, relres = core.paradiag_solve(N, lam, V, Vinv, om, fhat, tol=tol)
    return u, fhat, iters, relres


@pytest.mark.parametrize("fft", [1, 0])
@pytest.mark.parametrize("N,n,alpha", [(15, 4, 1e-2), (63, 16, 1e-3), (127, 8, 1e-3), (31, 128, 1e-3),
                                       (31, 2, 0.5)])
def test_transforms_fp64(N, n, alpha, fft):
    """FP64 time transforms, the Gamma-weighted FFTs of the alpha-circulant V (fft = 1) and
    the dense products (fft = 0), against the oracle's dense products."""
    rng = np.random.default_rng(N)
    c = api.alpha_circulant_context(N, n, 1.0 / n, alpha, fft_transforms=fft)
    lam, V, Vinv = core.alpha_circulant(n, 1.0 / n, alpha)
    f = rng.uniform(-1, 1, (n, N, N))
    u0 = inputs.sine_initial_value(N)
    g = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    c.pd_transform_forward(g, dev(f), dev(u0))
    fhat = core.assemble_rhs(N, n, 1.0 / n, f, u0)
    ref = core.time_transform(Vinv, fhat.reshape(n, -1)).reshape(n, N, N)
    assert rel_per_vector(host(g), ref) < 1e-13
    z = rng.uniform(-1, 1, (n, N, N)) + 1j * rng.uniform(-1, 1, (n, N, N))
    u = torch.full((n, N, N), 0.5, dtype=torch.float64, device="cuda")
    c.pd_transform_inverse(u, dev(z, torch.complex128), accumulate=True)
    ref = core.time_transform(V, z.reshape(n, -1)).real.reshape(n, N, N) + 0.5
    assert rel_per_vector(host(u), ref) < 1e-13


def test_allatonce_residual_fp64():
    N, n, tau, alpha = 31, 8, 1 / 8, 1e-3
    rng = np.random.default_rng(2)
    c = api.alpha_circulant_context(N, n, tau, alpha)
    u = rng.standard_normal((n, N, N))
    f = rng.standard_normal((n, N, N))
    u0 = rng.standard_normal((N, N))
    r = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    rn, fn = c.pd_allatonce_residual(r, dev(u), dev(f), dev(u0))
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    rno, fno, ro = core.allatonce_residual(N, n, tau, alpha, u, fhat, want_r=True)
    assert rel_per_vector(host(r), ro) < 1e-14 * 100
    assert abs(rn - rno) < 1e-12 * rno and abs(fn - fno) < 1e-12 * fno


@pytest.mark.parametrize("N,n,alpha", [(31, 4, 1e-2), (63, 16, 1e-3), (127, 8, 1e-3)])
def test_paradiag_fp64(N, n, alpha):
    tau = 1.0 / n
    f, u0 = inputs.paradiag_problem(N, n, seed=1)
    c = api.alpha_circulant_context(N, n, tau, alpha)
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    out = c.paradiag_solve(u, dev(f), dev(u0))
    uo, fhat, ito, rro = oracle_paradiag(N, n, tau, alpha, f, u0)
    assert np.array_equal(out["iters"], ito)
    assert np.all(out["relres"] <= 1e-10)
    uh = host(u)
    assert weighted_rel_err(uh, uo, alpha) < 1e-12
    rn, fn = core.allatonce_residual(N, n, tau, alpha, uh, fhat)
    rno, _ = core.allatonce_residual(N, n, tau, alpha, uo, fhat)
    noise = residual_rounding(N, n, tau, alpha, uh, fhat) / fn
    assert abs(out["relres_allatonce"] - rn / fn) <= 1e-3 * rn / fn + noise
    assert np.linalg.norm(uh - uo) <= residual_error_bound(N, n, alpha, rn / fn, rno / fn, fn)
    assert out["imag_max"] < 1e-10 * np.max(np.abs(uo)) / alpha


@pytest.mark.parametrize("N,n,alpha", [(63, 16, 1e-3), (127, 8, 1e-3), (255, 16, 1e-3)])
def test_paradiag_precision_form(N, n, alpha):
    """FP32 cycles inside FP64 refinement reach ||fhat - A u|| / ||fhat|| <= 1e-10 on eq. (1)."""
    tau = 1.0 / n
    f, u0 = inputs.paradiag_problem(N, n, seed=1)
    c = api.alpha_circulant_context(N, n, tau, alpha, precision=1)
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    out = c.paradiag_solve(u, dev(f), dev(u0))
    uh = host(u)
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    rn, fn = core.allatonce_residual(N, n, tau, alpha, uh, fhat)
    assert rn / fn <= 1e-10 and out["relres_allatonce"] <= 1e-10
    noise = residual_rounding(N, n, tau, alpha, uh, fhat) / fn
    assert abs(out["relres_allatonce"] - rn / fn) <= 1e-3 * rn / fn + noise
    assert 1 <= out["refine_steps"] <= 10
    uo, _, _, _ = oracle_paradiag(N, n, tau, alpha, f, u0, tol=1e-12)
    rno, _ = core.allatonce_residual(N, n, tau, alpha, uo, fhat)
    assert np.linalg.norm(uh - uo) <= residual_error_bound(N, n, alpha, rn / fn, rno / fn, fn)
    assert weighted_rel_err(uh, uo, alpha) < 1e-8


def test_paradiag_host_api_matches_device():
    N, n = 63, 8
    f, u0 = inputs.paradiag_problem(N, n, seed=4)
    c = api.alpha_circulant_context(N, n, 1.0 / n, 1e-3)
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    out = c.paradiag_solve(u, dev(f), dev(u0))
    uh = torch.empty(n, N, N, dtype=torch.float64).pin_memory()
    fh = torch.from_numpy(f).pin_memory()
    u0h = torch.from_numpy(u0).pin_memory()
    out2 = c.paradiag_solve_host(uh, fh, u0h)
    assert np.array_equal(uh.numpy(), host(u))
    assert np.array_equal(out["iters"], out2["iters"])


def test_paradiag_without_V_is_a_state_error():
    c = api.Context(15, 2, [1.0, 2.0])
    u = torch.empty(2, 15, 15, dtype=torch.float64, device="cuda")
    with pytest.raises(api.PDError) as e:
        c.paradiag_solve(u, u.clone())
    assert e.value.status == "PD_ERR_STATE"


@pytest.mark.parametrize("path", ["fft", "tc", "cuda_cores"])
@pytest.mark.parametrize("N,n", [(127, 16), (255, 64), (255, 5), (127, 128)])
def test_transforms_fp32(path, N, n):
    """FP32 context: Gamma-weighted FFTs (path fft), TF32x3 tcgen05 products (tc) and FP32
    CUDA-core products against the FP64 oracle: relative error per shift vector of a few
    1e-7 (TF32x3 keeps about 21 bits per product; fhat is rounded to FP32 first)."""
    alpha = 1e-3
    rng = np.random.default_rng(N + n)
    c = api.alpha_circulant_context(N, n, 1.0 / n, alpha, precision=1,
                                    tensor_transforms=int(path == "tc"), fft_transforms=int(path == "fft"))
    lam, V, Vinv = core.alpha_circulant(n, 1.0 / n, alpha)
    f = rng.uniform(-1, 1, (n, N, N))
    u0 = inputs.sine_initial_value(N)
    g = torch.empty(n, N, N, dtype=torch.complex64, device="cuda")
    c.pd_transform_forward(g, dev(f), dev(u0))
    fhat = core.assemble_rhs(N, n, 1.0 / n, f, u0)
    ref = core.time_transform(Vinv, fhat.reshape(n, -1)).reshape(n, N, N)
    assert rel_per_vector(host(g), ref) < 2e-6
    z = (rng.uniform(-1, 1, (n, N, N)) + 1j * rng.uniform(-1, 1, (n, N, N))).astype(np.complex64)
    u = torch.full((n, N, N), 0.25, dtype=torch.float64, device="cuda")
    c.pd_transform_inverse(u, dev(z, torch.complex64), accumulate=True)
    ref = core.time_transform(V, z.astype(np.complex128).reshape(n, -1)).real.reshape(n, N, N) + 0.25
    g_w = (alpha ** (np.arange(n) / n))[:, None, None]
    err = np.linalg.norm(g_w * (host(u) - ref)) / np.linalg.norm(g_w * ref)
    assert err < 2e-6


def converged_iterate(N, n, tau, alpha, fhat, steps=3):
    """u with ||fhat - A u|| / ||fhat|| near the FP64 floor: oracle ParaDIAG steps refined
    with the oracle's own residual."""
    lam, V, Vinv = core.alpha_circulant(n, tau, alpha)
    om = lfa.omega_table(lam, N, mode="lfa")
    u = np.zeros_like(fhat)
    for _ in range(steps):
        _, _, r = core.allatonce_residual(N, n, tau, alpha, u, fhat, want_r=True)
        d, _, _, _ = core.paradiag_solve(N, lam, V, Vinv, om, r, tol=1e-12)
        u += d
    return u


@pytest.mark.parametrize("fx", [1, 0])
@pytest.mark.parametrize("N,n,alpha", [(127, 8, 1e-3), (255, 16, 1e-2), (63, 5, 0.3), (31, 4, 1e-3)])
def test_refinement_residual32(fx, N, n, alpha):
    """The FP32 residual the refinement hands to the forward transform, element by element
    against the oracle's long-double residual, on a random and on a converged u (N = 31:
    every warp tile touches the grid's edge; N = 63: one column of interior tiles).  Without
    FP64 arithmetic (fx = 1) the error bound is the FP32 rounding of r plus 2^-43 of the
    terms and the fixed-point truncation ih2 2^-54 max|u_k| — far below the FP64 rounding of
    the formula (4 eps of ih2 (4|u| + sum|nb|)), which bounds fx = 0."""
    tau = 1.0 / n
    h = 1.0 / (N + 1)
    ih2 = 1.0 / h ** 2
    f, u0 = inputs.paradiag_problem(N, n, seed=7)
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    c = api.alpha_circulant_context(N, n, tau, alpha, precision=1, fx_residual=fx)
    rng = np.random.default_rng(N + n)
    for u in (rng.standard_normal((n, N, N)), converged_iterate(N, n, tau, alpha, fhat)):
        r32 = torch.empty(n, N, N, dtype=torch.float32, device="cuda")
        rn, fn = c.pd_allatonce_residual32(r32, dev(u), dev(f), dev(u0))
        r = host(r32).astype(np.float64)
        rn_ld, r_ld = core.allatonce_residual_ld(N, n, tau, alpha, u, fhat)
        a = np.abs(u)
        nb = np.zeros_like(u)
        nb[:, 1:, :] += u[:, :-1, :]
        nb[:, :-1, :] += u[:, 1:, :]
        nb[:, :, 1:] += u[:, :, :-1]
        nb[:, :, :-1] += u[:, :, 1:]
        anb = np.zeros_like(a)
        anb[:, 1:, :] += a[:, :-1, :]
        anb[:, :-1, :] += a[:, 1:, :]
        anb[:, :, 1:] += a[:, :, :-1]
        anb[:, :, :-1] += a[:, :, 1:]
        prev = np.roll(a, 1, axis=0)
        prev[0] *= alpha
        if fx:
            T = np.abs(fhat) + (a + prev) / tau + ih2 * np.abs(4 * u - nb)
            umax = np.max(a.reshape(n, -1), axis=1)[:, None, None]
            tol = 2.0 ** -24 * np.abs(r_ld) + 2.0 ** -43 * T + ih2 * 2.0 ** -54 * umax
        else:
            T = np.abs(fhat) + (a + prev) / tau + ih2 * (4 * a + anb)
            tol = 2.0 ** -24 * np.abs(r_ld) + 4 * np.finfo(float).eps * T
        assert np.all(np.abs(r - r_ld) <= tol)
        assert abs(rn - rn_ld) <= 1e-5 * rn_ld + np.linalg.norm(tol)
        assert fn == pytest.approx(np.linalg.norm(fhat), rel=1e-5)


def fx_bound(N, n, tau, alpha, u, fhat, r_ld):
    """Element bound of the fixed-point residual (as in test_refinement_residual32): FP32
    rounding of r, 2^-43 of the terms, the truncation ih2 2^-54 max|u_k|."""
    ih2 = float(N + 1) ** 2
    a = np.abs(u)
    nb = np.zeros_like(u)
    nb[:, 1:, :] += u[:, :-1, :]
    nb[:, :-1, :] += u[:, 1:, :]
    nb[:, :, 1:] += u[:, :, :-1]
    nb[:, :, :-1] += u[:, :, 1:]
    prev = np.roll(a, 1, axis=0)
    prev[0] *= alpha
    T = np.abs(fhat) + (a + prev) / tau + ih2 * np.abs(4 * u - nb)
    umax = np.max(a.reshape(n, -1), axis=1)[:, None, None]
    return 2.0 ** -24 * np.abs(r_ld) + 2.0 ** -43 * T + ih2 * 2.0 ** -54 * umax


@pytest.mark.parametrize("N,n,alpha", [(127, 8, 1e-3), (255, 16, 1e-2), (63, 5, 0.3), (31, 3, 0.1)])
def test_refinement_residual32_transposed(N, n, alpha):
    """The same residual for the adjoint's transposed time matrix, whose kernel walks the
    time steps downwards: B^T = J B J with J the reversal of the time steps, so the
    residual of (B^T x I + I x A) u = f is J times the oracle's long-double residual of
    the forward system for J u and J f."""
    tau = 1.0 / n
    c = api.alpha_circulant_context(N, n, tau, alpha, precision=1)
    adj = c.adjoint()
    rng = np.random.default_rng(3 * N + n)
    f = rng.standard_normal((n, N, N))
    for u in (rng.standard_normal((n, N, N)),
              np.cumsum(rng.standard_normal((n, N, N)), axis=0) * 1e-3 + 1.0):
        r32 = torch.empty(n, N, N, dtype=torch.float32, device="cuda")
        rn, fn = adj.pd_allatonce_residual32(r32, dev(u), dev(f), None)
        r = host(r32).astype(np.float64)
        ur, fr = np.ascontiguousarray(u[::-1]), np.ascontiguousarray(f[::-1])
        rn_ld, r_ld = core.allatonce_residual_ld(N, n, tau, alpha, ur, fr)
        tol = fx_bound(N, n, tau, alpha, ur, fr, r_ld)
        assert np.all(np.abs(r[::-1] - r_ld) <= tol)
        assert abs(rn - rn_ld) <= 1e-5 * rn_ld + np.linalg.norm(tol)
        assert fn == pytest.approx(np.linalg.norm(f), rel=1e-5)


@pytest.mark.parametrize("precision,n,out_mem", [(1, 8, "pinned"), (0, 8, "pinned"), (1, 8, "pageable"),
                                                   (1, 5, "pinned")])
def test_paradiag_host_batch_pipelined(precision, n, out_mem):
    """paradiag_solve_host_batch: three independent steps with host buffers, copies of the
    neighbouring steps overlapping each solve, each result identical to paradiag_solve on
    the same input.  u goes out by the streaming copy kernel into pinned memory (n = 8), by
    the copy engine into pageable memory and for a size that is not a multiple of 16 bytes
    (n = 5)."""
    N, tau, alpha = 63, 1.0 / 8, 1e-3
    c = api.alpha_circulant_context(N, n, tau, alpha, precision=precision)
    probs = [inputs.paradiag_problem(N, n, seed=20 + k) for k in range(3)]
    fs = [torch.from_numpy(f).pin_memory() for f, _ in probs]
    u0s = [torch.from_numpy(u0).pin_memory() for _, u0 in probs]
    if out_mem == "pinned":
        us = [torch.empty_like(fs[0]).pin_memory() for _ in range(3)]
    else:
        us = [torch.empty_like(fs[0]) for _ in range(3)]
        assert not us[0].is_pinned()
    outs = c.paradiag_solve_host_batch(us, fs, u0s)
    for (f, u0), uh, out in zip(probs, us, outs):
        ud = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
        ref = c.paradiag_solve(ud, dev(f), dev(u0))
        assert np.array_equal(uh.numpy(), host(ud))
        assert np.array_equal(out["iters"], ref["iters"])
        assert out["relres_allatonce"] == ref["relres_allatonce"]


@pytest.mark.parametrize("n", [100, 128])
def test_transforms_tc_wide(n):
    """The tensor-core transforms for 64 < n <= 128 (forward rows and inverse K split over two
    CTAs, the inverse's halves summed in a two-CTA cluster) against the oracle's dense
    products, on a general V (the alpha-circulant B diagonalised by the library, so the
    FFT route does not apply): relative error per shift vector a few 1e-7 (TF32x3)."""
    N, alpha = 127, 1e-2
    B = api.pd_alpha_circulant(n, 1.0 / n, alpha)[0]
    c = api.dense_B_context(B, N, None, precision=1)
    lam, V, Vinv = api.pd_diagonalize(B)  # the library's eigenvectors: those c uses
    rng = np.random.default_rng(n)
    f = rng.uniform(-1, 1, (n, N, N))
    g = torch.empty(n, N, N, dtype=torch.complex64, device="cuda")
    c.pd_transform_forward(g, dev(f))
    ref = core.time_transform(Vinv, f.reshape(n, -1)).reshape(n, N, N)
    assert rel_per_vector(host(g), ref) < 2e-6
    z = (rng.uniform(-1, 1, (n, N, N)) + 1j * rng.uniform(-1, 1, (n, N, N))).astype(np.complex64)
    u = torch.full((n, N, N), 0.25, dtype=torch.float64, device="cuda")
    c.pd_transform_inverse(u, dev(z, torch.complex64), accumulate=True)
    ref = core.time_transform(V, z.astype(np.complex128).reshape(n, -1)).real.reshape(n, N, N) + 0.25
    assert np.linalg.norm(host(u) - ref) / np.linalg.norm(ref) < 2e-6


def test_paradiag_dense_B_tensor_cores_n128():
    """The precision form through the tensor-core transforms at n = 128 (B given alone: the
    alpha-circulant matrix, diagonalised by the library): the oracle's FP64 residual of
    eq. (1) reaches 1e-10."""
    N, n, alpha = 255, 128, 1e-3
    tau = 1.0 / n
    B, _, _, _, c0 = api.pd_alpha_circulant(n, tau, alpha)
    c = api.dense_B_context(B, N, c0, precision=1)
    f, u0 = inputs.paradiag_problem(N, n, seed=3)
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    out = c.paradiag_solve(u, dev(f), dev(u0))
    assert out["relres_allatonce"] <= 1e-10 and out["imag_max"] == -1.0
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    rn, fn = core.allatonce_residual(N, n, tau, alpha, host(u), fhat)
    assert rn / fn <= 1e-10
