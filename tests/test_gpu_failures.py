"""Failure paths and convergence histories through the C ABI.

Failures are made on the host only (no kernel is made to fault, trap or hang): a
NaN placed in a right-hand side must come back as PD_ERR_NAN from every solve entry point,
in both precisions, and the same context must then solve clean data as before.  The
per-shift residual history of an FP64 shifted solve is compared with the oracle's history
cycle by cycle (the relative residual of Sec. 3's stopping test)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core, lfa  # noqa: E402
from paper_2203_11154_gb300 import api, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_stream(torch.cuda.Stream())


def _expect_nan(fn):
    with pytest.raises(api.PDError) as e:
        fn()
    assert e.value.status == "PD_ERR_NAN", e.value


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_in_source_paradiag_solve(precision):
    N, n, tau, alpha = 63, 16, 1.0 / 16, 1e-2
    c = api.alpha_circulant_context(N, n, tau, alpha, precision=precision)
    f, u0 = inputs.paradiag_problem(N, n, seed=1)
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    bad = f.copy()
    bad[3, 10, 20] = np.nan
    _expect_nan(lambda: c.paradiag_solve(u, torch.from_numpy(bad).cuda(), torch.from_numpy(u0).cuda()))
    out = c.paradiag_solve(u, torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda())
    assert out["status"] == "PD_OK"
    if precision == 1:
        assert out["relres_allatonce"] <= 1e-10
    else:
        assert out["relres_shift_max"] <= 1e-10
    c.destroy()


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_in_rhs_shifted_solves(precision):
    N, n = 63, 16
    lam = api.pd_shifts_alpha_circulant(n, 1.0 / 16, 1e-2)[0]
    b = inputs.shifted_problem(N, n, seed=0)
    bad = b.copy()
    bad[5, 30, 31] = complex(np.inf, 0.0)
    c = api.Context(N, n, lam, cfg=api.config(precision=precision))
    ct, nt = (torch.complex128, np.complex128) if precision == 0 else (torch.complex64, np.complex64)
    z = torch.empty(n, N, N, dtype=ct, device="cuda")
    _expect_nan(lambda: c.shifted_solve_batched(z, torch.from_numpy(bad.astype(nt)).cuda()))
    it, rr = c.shifted_solve_batched(z, torch.from_numpy(b.astype(nt)).cuda(), raise_on_noconv=False)
    assert np.all(np.isfinite(rr)) and np.all(it > 0)
    if precision == 1:
        z64 = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
        _expect_nan(lambda: c.shifted_solve_refined(z64, torch.from_numpy(bad).cuda()))
        it, rr = c.shifted_solve_refined(z64, torch.from_numpy(b).cuda())
        assert np.all(rr <= 1e-10)
    c.destroy()


def test_nan_in_one_instance_of_a_batch():
    probs = inputs.uneven_problem((31, 63), (4, 8), seed=2)
    bt = api.Batch([p[0] for p in probs], [p[1] for p in probs], api.config(precision=1))
    bs = [torch.from_numpy(p[2]).cuda() for p in probs]
    zs = [torch.empty_like(b) for b in bs]
    bad = [b.clone() for b in bs]
    bad[1][2, 7, 7] = complex(np.nan, 0.0)
    _expect_nan(lambda: bt.solve(zs, bad))
    out = bt.solve(zs, bs)
    assert all(np.all(rr <= 1e-10) for _, rr in out)
    bt.destroy()


def test_cycle_history_matches_oracle():
    """FP64 shifted solve: relres before the first cycle (1) and after each cycle, per shift,
    against the oracle's own history of the same solve."""
    N, n = 63, 16
    lam = api.pd_shifts_alpha_circulant(n, 1.0 / 16, 1e-2)[0]
    b = inputs.shifted_problem(N, n, seed=0)
    c = api.Context(N, n, lam, cfg=api.config(precision=0))
    z = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    it, rr = c.shifted_solve_batched(z, torch.from_numpy(b).cuda())
    hist, outer = c.history()
    om = lfa.omega_table(lam, N, mode="lfa")
    for j in range(n):
        _, ito, _, ho = core.shifted_solve(N, lam[j], om[j], b[j], tol=1e-10)
        assert it[j] == ito and hist[j].size == ito + 1
        assert abs(hist[j][0] - 1.0) <= 1e-14
        assert np.all(np.abs(hist[j] - ho) <= 1e-8 * ho + 1e-15)
    lines = c.history_jsonl().splitlines()
    assert len(lines) == n + 1
    c.destroy()


def test_refinement_history():
    """Precision form: the relative residual of eq. (1) after each refinement step decreases
    and its last entry is the reported one."""
    N, n, tau, alpha = 127, 16, 1.0 / 16, 1e-3
    c = api.alpha_circulant_context(N, n, tau, alpha, precision=1)
    f, u0 = inputs.paradiag_problem(N, n, seed=1)
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    out = c.paradiag_solve(u, torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda())
    _, outer = c.history()
    assert outer.size == out["refine_steps"]
    assert outer[-1] == out["relres_allatonce"] and outer[-1] <= 1e-10
    assert np.all(np.diff(outer) < 0)
    c.destroy()


@pytest.mark.parametrize("scale", [1e-15, 1e20])
def test_precision_form_does_not_depend_on_the_data_scale(scale):
    """The FP32 solves inside the FP64 refinement see right-hand sides scaled by powers of two
    to unit size, so a source and initial value scaled by 1e-15 or 1e20 still reach the
    oracle's relative residual of eq. (1) <= 1e-10 (the solve of eq. (1) is linear)."""
    N, n, tau, alpha = 127, 16, 1.0 / 16, 1e-3
    c = api.alpha_circulant_context(N, n, tau, alpha, precision=1)
    f, u0 = inputs.paradiag_problem(N, n, seed=1)
    f = f * scale
    u0 = u0 * scale
    u = torch.empty(n, N, N, dtype=torch.float64, device="cuda")
    out = c.paradiag_solve(u, torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda())
    assert out["relres_allatonce"] <= 1e-10
    torch.cuda.synchronize()
    fhat = core.assemble_rhs(N, n, tau, f, u0)
    rn, fn = core.allatonce_residual(N, n, tau, alpha, u.cpu().numpy(), fhat)
    assert rn / fn <= 1e-10
    assert abs(rn / fn - out["relres_allatonce"]) <= 0.05 * rn / fn + 1e-13
    c.destroy()


@pytest.mark.parametrize("scale", [1e-15, 1e20])
def test_refined_shifted_solve_does_not_depend_on_the_data_scale(scale):
    """shifted_solve_refined with right-hand sides scaled by 1e-15 or 1e20: every shift reaches
    the oracle's FP64 relative residual <= 1e-10."""
    N, n = 127, 16
    lam = api.pd_shifts_alpha_circulant(n, 1.0 / 16, 1e-2)[0]
    b = inputs.shifted_problem(N, n, seed=0) * scale
    c = api.Context(N, n, lam, cfg=api.config(precision=1))
    z = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    it, rr = c.shifted_solve_refined(z, torch.from_numpy(b).cuda())
    assert np.all(rr <= 1e-10)
    torch.cuda.synchronize()
    zh = z.cpu().numpy()
    for j in range(n):
        r = core.residual(N, lam[j], b[j], zh[j])
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[j])
    c.destroy()


@pytest.mark.parametrize("fx", [0, 1])
@pytest.mark.parametrize("N,n", [(127, 8), (255, 4), (31, 3)])
def test_shifted_residual32_against_long_double_oracle(fx, N, n):
    """The FP32 residual of eq. (2) the refined shifted solves hand to the multigrid, element
    by element against the oracle's long-double residual, on a random z and on a converged
    one (N = 31: every warp tile touches the grid's edge).  Without FP64 arithmetic (fx = 1) the bound is the FP32 rounding of r plus 2^-43
    of the terms and the fixed-point truncation ih2 2^-54 max|z_j| per component; the FP64
    formula (fx = 0) is bound by its rounding, 4 eps of the terms, and its FP32 output is
    truncated (not rounded) to 24 bits: 2^-23 |r|."""
    lam = inputs.random_shifts(np.random.default_rng(N), n)
    b = inputs.complex_rhs(np.random.default_rng(N + 1), n, N)
    c = api.Context(N, n, lam, cfg=api.config(precision=1, fx_residual=fx))
    ih2 = float(N + 1) ** 2
    z_conv = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    c.shifted_solve_refined(z_conv, torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    rng = np.random.default_rng(N + 2)
    for z in (inputs.complex_rhs(rng, n, N), z_conv.cpu().numpy()):
        r32 = torch.empty(n, N, N, dtype=torch.complex64, device="cuda")
        norms = c.pd_shifted_residual32(r32, torch.from_numpy(z).cuda(), torch.from_numpy(b).cuda())
        r = r32.cpu().numpy().astype(np.complex128)
        for j in range(n):
            r_ld = core.residual_ld(N, lam[j], b[j], z[j])
            for part in (np.real, np.imag):
                zc = part(z[j])
                nb = np.zeros_like(zc)
                nb[1:, :] += zc[:-1, :]
                nb[:-1, :] += zc[1:, :]
                nb[:, 1:] += zc[:, :-1]
                nb[:, :-1] += zc[:, 1:]
                anb = np.zeros_like(zc)
                az = np.abs(zc)
                anb[1:, :] += az[:-1, :]
                anb[:-1, :] += az[1:, :]
                anb[:, 1:] += az[:, :-1]
                anb[:, :-1] += az[:, 1:]
                lz = np.abs(lam[j]) * np.abs(z[j])
                if fx:
                    T = np.abs(part(b[j])) + lz + ih2 * np.abs(4 * zc - nb)
                    tol = 2.0 ** -24 * np.abs(part(r_ld)) + 2.0 ** -43 * T + ih2 * 2.0 ** -54 * np.max(az)
                else:
                    T = np.abs(part(b[j])) + lz + ih2 * (4 * az + anb)
                    tol = 2.0 ** -23 * np.abs(part(r_ld)) + 4 * np.finfo(float).eps * T
                assert np.all(np.abs(part(r[j]) - part(r_ld)) <= tol)
            assert norms[j] == pytest.approx(np.linalg.norm(r[j]), rel=1e-5)
    c.destroy()
