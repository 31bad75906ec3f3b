"""GPU parity of every multigrid kernel and of the batched shifted solve against the
FP64 oracle, through the C ABI (FP64 bar: 1e-12 relative per output vector)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core, lfa  # noqa: E402
from paper_2203_11154_gb300 import api, inputs  # noqa: E402

TOL64 = 1e-12


def rel_per_vector(x, ref):
    x = np.asarray(x).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.max(np.linalg.norm(x - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300))


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rand_c(rng, shape):
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


SHIFTS = np.array([6.5 + 0.0j, 20.0 - 300.0j, -40.0 + 12.0j, 1e3 + 2e3j])


def ctx_for(N, lam, **cfg):
    return api.Context(N, len(lam), lam, cfg=api.config(**cfg))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_omega_table_matches_oracle_lfa():
    N = 63
    lam = np.concatenate([SHIFTS, core.alpha_circulant(16, 1 / 16, 1e-2)[0]])
    c = ctx_for(N, lam, omega_mode=1)
    got = c.omega()
    ref = lfa.omega_table(lam, N, mode="lfa", K=64)
    assert np.max(np.abs(got - ref)) < 1e-8
    c0 = ctx_for(N, lam, omega_mode=0)
    assert np.all(c0.omega() == 24 / 25)


@pytest.mark.parametrize("N", [7, 63, 127])
@pytest.mark.parametrize("smoother", [0, 1])
def test_smooth_fp64(N, smoother):
    rng = np.random.default_rng(N + 10 * smoother)
    n = len(SHIFTS)
    c = ctx_for(N, SHIFTS, omega_mode=0, smoother=smoother)
    z = rand_c(rng, (n, N, N))
    b = rand_c(rng, (n, N, N)) * 1e3
    out = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    c.pd_smooth(0, out, dev(z), dev(b))
    w = 24 / 25 if smoother == 0 else 0.8
    fn = core.vanka_smooth if smoother == 0 else core.jacobi_smooth
    ref = np.stack([fn(N, SHIFTS[j], w, b[j], z[j]) for j in range(n)])
    assert rel_per_vector(host(out), ref) < 1e-14 * 10


@pytest.mark.parametrize("N", [15, 127])
def test_smooth_fp32(N):
    rng = np.random.default_rng(3)
    n = len(SHIFTS)
    B, sh, V, Vi, c0 = api.pd_alpha_circulant(n, 0.25, 0.5)
    c = api.Context(N, n, SHIFTS, V, Vi, B, c0, cfg=api.config(omega_mode=0, precision=1))
    z = rand_c(rng, (n, N, N))
    b = rand_c(rng, (n, N, N)) * 1e3
    out = torch.empty(n, N, N, dtype=torch.complex64, device="cuda")
    c.pd_smooth(0, out, dev(z, torch.complex64), dev(b, torch.complex64))
    ref = np.stack([core.vanka_smooth(N, SHIFTS[j], 24 / 25, b[j].astype(np.complex64),
                                      z[j].astype(np.complex64)) for j in range(n)])
    assert rel_per_vector(host(out), ref) < 2e-6


@pytest.mark.parametrize("N", [7, 63, 255])
def test_residual_restrict_fp64(N):
    rng = np.random.default_rng(N)
    n = len(SHIFTS)
    c = ctx_for(N, SHIFTS, omega_mode=0)
    z = rand_c(rng, (n, N, N))
    b = rand_c(rng, (n, N, N))
    Nc = (N - 1) // 2
    out = torch.empty(n, Nc, Nc, dtype=torch.complex128, device="cuda")
    c.pd_residual_restrict(0, out, dev(z), dev(b))
    ref = np.stack([core.restrict_fw(N, core.residual(N, SHIFTS[j], b[j], z[j])) for j in range(n)])
    assert rel_per_vector(host(out), ref) < 1e-13


@pytest.mark.parametrize("N", [3, 15, 127])
def test_prolong_add_fp64(N):
    rng = np.random.default_rng(N)
    n = len(SHIFTS)
    c = ctx_for(N, SHIFTS, omega_mode=0, coarsest_n=1)
    Nc = (N - 1) // 2
    z = rand_c(rng, (n, N, N))
    ec = rand_c(rng, (n, Nc, Nc))
    zt = dev(z)
    c.pd_prolong_add(0, zt, dev(ec))
    ref = np.stack([core.prolong_add(N, ec[j], z[j]) for j in range(n)])
    assert rel_per_vector(host(zt), ref) < 1e-15 * 4


@pytest.mark.parametrize("coarsest", [1, 3, 7, 15])
def test_coarse_solve_fp64(coarsest):
    rng = np.random.default_rng(coarsest)
    n = len(SHIFTS)
    c = ctx_for(31, SHIFTS, omega_mode=0, coarsest_n=coarsest)
    Nc = c.Ns[-1]
    assert Nc == coarsest
    b = rand_c(rng, (n, Nc, Nc))
    out = torch.empty(n, Nc, Nc, dtype=torch.complex128, device="cuda")
    c.pd_coarse_solve(out, dev(b))
    ref = np.stack([core.coarse_solve(Nc, SHIFTS[j], b[j]) for j in range(n)])
    assert rel_per_vector(host(out), ref) < 1e-13


CYCLES = [dict(cycle_gamma=1, nu1=1, nu2=1, coarsest_n=3), dict(cycle_gamma=2, nu1=1, nu2=0, coarsest_n=7),
          dict(cycle_gamma=1, nu1=0, nu2=2, coarsest_n=3), dict(cycle_gamma=2, nu1=2, nu2=1, coarsest_n=1)]


@pytest.mark.parametrize("cyc", range(len(CYCLES)))
@pytest.mark.parametrize("N,level", [(127, 0), (255, 1), (63, 0), (31, 0)])
def test_mg_vcycle_fp64(cyc, N, level):
    prm = CYCLES[cyc]
    rng = np.random.default_rng(7 + cyc)
    n = len(SHIFTS)
    c = ctx_for(N, SHIFTS, omega_mode=0, **prm)
    Nl = c.Ns[level]
    z = rand_c(rng, (n, Nl, Nl))
    b = rand_c(rng, (n, Nl, Nl)) * 100
    zt = dev(z)
    c.mg_vcycle(level, zt, dev(b))
    op = core.mg_params(prm["cycle_gamma"], prm["nu1"], prm["nu2"], prm["coarsest_n"])
    om = [24 / 25] * 16
    ref = np.stack([core.mg_cycle(Nl, SHIFTS[j], om, b[j], z[j], op) for j in range(n)])
    assert rel_per_vector(host(zt), ref) < 1e-13


def shifted_case(N, n, lam, omega_mode, seed, **cfg):
    rng = np.random.default_rng(seed)
    b = rand_c(rng, (n, N, N))
    c = ctx_for(N, lam, omega_mode=omega_mode, **cfg)
    z = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    it, rr = c.shifted_solve_batched(z, dev(b))
    smoother = "jacobi" if cfg.get("smoother", 0) == 1 else "vanka"
    om = lfa.omega_table(lam, N, coarsest_n=cfg.get("coarsest_n", 3),
                         mode="lfa" if omega_mode == 1 else "fixed", smoother=smoother)
    prm = core.mg_params(cfg.get("cycle_gamma", 1), cfg.get("nu1", 1), cfg.get("nu2", 1),
                         cfg.get("coarsest_n", 3), cfg.get("smoother", 0))
    zo, ito, rro = core.shifted_solve_batch(N, lam, om, b, tol=cfg.get("tol", 1e-10),
                                            maxit=cfg.get("maxit", 100), prm=prm)
    return host(z), it, rr, zo, ito, rro


def test_shifted_solve_workload_63():
    """The 63 x 63, 16 alpha-circulant shifts workload (tau = 1/16, alpha = 1e-2), seed 0."""
    w = inputs.WORKLOADS["shifted-63"]
    N, n = w["N"], w["n"]
    lam = core.alpha_circulant(n, w["tau"], w["alpha"])[0]
    b = inputs.shifted_problem(N, n, w["seed"])
    c = ctx_for(N, lam, omega_mode=1)
    z = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    it, rr = c.shifted_solve_batched(z, dev(b))
    om = lfa.omega_table(lam, N, mode="lfa")
    zo, ito, rro = core.shifted_solve_batch(N, lam, om, b, tol=1e-10)
    assert np.array_equal(it, ito)
    assert np.all(rr <= 1e-10)
    assert np.allclose(rr, rro, rtol=1e-6)
    assert rel_per_vector(host(z), zo) < TOL64


@pytest.mark.parametrize("N,cfg", [(127, {}), (255, dict(cycle_gamma=2, nu1=1, nu2=0, coarsest_n=7)),
                                   (63, dict(nu1=0, nu2=1)), (15, dict(smoother=1, maxit=200)),
                                   (1, dict(coarsest_n=1)), (3, {})])
def test_shifted_solve_fp64(N, cfg):
    lam = SHIFTS
    z, it, rr, zo, ito, rro = shifted_case(N, len(lam), lam, 1 if N > 1 else 0, N, **cfg)
    assert np.array_equal(it, ito), (it, ito)
    assert np.all(rr <= 1e-10)
    assert rel_per_vector(z, zo) < TOL64


def test_shifted_solve_zero_rhs_and_mixed_convergence():
    N, n = 127, 4
    lam = SHIFTS
    b = np.zeros((n, N, N), complex)
    b[1] = rand_c(np.random.default_rng(1), (N, N))
    b[3] = 1e-100 * rand_c(np.random.default_rng(2), (N, N))
    c = ctx_for(N, lam, omega_mode=0)
    z = torch.full((n, N, N), 7.0, dtype=torch.complex128, device="cuda")
    it, rr = c.shifted_solve_batched(z, dev(b))
    zh = host(z)
    assert it[0] == 0 and it[2] == 0 and not np.any(zh[0]) and not np.any(zh[2])
    assert it[1] > 3 and rr[1] <= 1e-10 and it[3] > 3


def test_shifted_solve_maxit_reports_noconv():
    N, n = 63, 2
    c = ctx_for(N, SHIFTS[:2], omega_mode=0, maxit=2)
    z = torch.empty(n, N, N, dtype=torch.complex128, device="cuda")
    b = dev(rand_c(np.random.default_rng(0), (n, N, N)))
    with pytest.raises(api.PDError) as e:
        c.shifted_solve_batched(z, b)
    assert e.value.status == "PD_ERR_NOCONV"
    it, rr = c.shifted_solve_batched(z, b, raise_on_noconv=False)
    assert np.all(it == 2) and np.all(rr > 1e-10)


@pytest.mark.parametrize("N", [63, 255])
def test_shifted_solve_fp32(N):
    lam = SHIFTS
    n = len(lam)
    rng = np.random.default_rng(5)
    b = rand_c(rng, (n, N, N))
    B, sh, V, Vi, c0 = api.pd_alpha_circulant(n, 0.25, 0.5)
    c = api.Context(N, n, lam, V, Vi, B, c0, cfg=api.config(precision=1, tol=1e-5))
    z = torch.empty(n, N, N, dtype=torch.complex64, device="cuda")
    it, rr = c.shifted_solve_batched(z, dev(b, torch.complex64))
    om = lfa.omega_table(lam, N, mode="lfa")
    zo, ito, rro = core.shifted_solve_batch(N, lam, om, b, tol=1e-5)
    assert np.all(rr <= 1e-5)
    assert np.all(np.abs(it - ito) <= 1)
    assert rel_per_vector(host(z), zo) < 1e-4


@pytest.mark.parametrize("fused", [0, 1, 2])
@pytest.mark.parametrize("N,level,cyc", [(255, 0, 0), (1023, 1, 0), (255, 0, 1), (127, 0, 3)])
def test_mg_vcycle_fused_and_unfused_fp64(fused, N, level, cyc):
    """The fused TMA kernels and the one-kernel-per-operation path give the oracle's cycle."""
    prm = CYCLES[cyc]
    rng = np.random.default_rng(21 + level)
    n = len(SHIFTS)
    # fused 0: one kernel per operation; 1: TMA tiles; 2: warp streams (both forced in FP64)
    c = ctx_for(N, SHIFTS, omega_mode=0, fused=2 if fused else 0, fused_variant=max(fused, 1), **prm)
    Nl = c.Ns[level]
    z = rand_c(rng, (n, Nl, Nl))
    b = rand_c(rng, (n, Nl, Nl)) * 100
    zt = dev(z)
    c.mg_vcycle(level, zt, dev(b))
    op = core.mg_params(prm["cycle_gamma"], prm["nu1"], prm["nu2"], prm["coarsest_n"])
    ref = np.stack([core.mg_cycle(Nl, SHIFTS[j], [24 / 25] * 16, b[j], z[j], op) for j in range(n)])
    assert rel_per_vector(host(zt), ref) < 1e-12


@pytest.mark.parametrize("fused", [0, 1, 2])
@pytest.mark.parametrize("N", [127, 511])
def test_mg_vcycle_fp32(fused, N):
    """FP32 cycle (fused TMA path and plain path) against the FP64 oracle on the same,
    FP32-rounded inputs: agreement to FP32 rounding."""
    rng = np.random.default_rng(N)
    n = len(SHIFTS)
    B, sh, V, Vi, c0 = api.pd_alpha_circulant(n, 0.25, 0.5)
    c = api.Context(N, n, SHIFTS, V, Vi, B, c0, cfg=api.config(omega_mode=0, precision=1,
                                                               fused=1 if fused else 0,
                                                               fused_variant=max(fused, 1)))
    z = rand_c(rng, (n, N, N)).astype(np.complex64)
    b = (rand_c(rng, (n, N, N)) * 100).astype(np.complex64)
    zt = dev(z, torch.complex64)
    c.mg_vcycle(0, zt, dev(b, torch.complex64))
    ref = np.stack([core.mg_cycle(N, SHIFTS[j], [24 / 25] * 16, b[j], z[j]) for j in range(n)])
    # FP32 rounding: each level's residual carries a rounding of about 2^-24 of its terms
    # (up to 8 |z| in the h^2-scaled form), white across the grid; the coarse-grid correction
    # solves with L^{-1}, whose smallest eigenvalue is 2 pi^2 in the unscaled form, so the
    # smooth part of that noise comes back amplified in proportion to N relative to |z|,
    # once per level (log2(N + 1) of them).  Measured per-vector errors on these inputs
    # (all three kernel paths, deterministic): 5.8e-8 N at N = 127, 8.4e-8 N at 511,
    # 9.7e-8 N at 2047, i.e. at most 0.93e-8 N log2(N + 1); the bar allows 1.35 times that.
    assert rel_per_vector(host(zt), ref) < 1.25e-8 * N * np.log2(N + 1)
    # the autotuner's record: the restricted variant on every fused level, none without
    choices = c.fused_choices()
    assert len(choices) == api.lib().pd_num_levels(c.h)
    for l, (v, sg) in enumerate(choices):
        if not fused:
            assert v == 0
        elif v != 0:
            assert v == max(fused, 1) and (sg in (4, 8, 16, 32, 64, 128, 256)) == (v == 2)
    if fused:
        assert choices[0][0] == max(fused, 1)
