"""Batched uneven form: independent shifted-system problems of different grid sizes and
shift counts solved together (pd_batch), and the FP64-refined shifted solve it uses in
precision 1.  FP64 multigrid against the oracle cycle for cycle; FP32 multigrid + FP64
refinement against the oracle's FP64 residual; CUDA-graph replay against launching
kernel by kernel; the full-size eight-instance workload on sampled shifts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core, lfa  # noqa: E402
from paper_2203_11154_gb300 import api, inputs  # noqa: E402

SMALL = dict(Ns=(31, 63, 63, 127), ns=(4, 8, 8, 16), seed=2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.complex128)


def rel_per_vector(x, ref):
    x = np.asarray(x).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.max(np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1))


def oracle_relres(N, lam, b, z):
    """||b - (lam I + A) z|| / ||b|| in FP64 by the oracle, and the rounding bound of
    evaluating it: 8 eps || |b| + (|lam| + 4/h^2)|z| + (1/h^2)(sum of |neighbours|) ||."""
    r = core.residual(N, lam, b, z)
    bn = np.linalg.norm(b)
    h = 1.0 / (N + 1)
    a = np.abs(z)
    nb = np.zeros_like(a)
    nb[1:, :] += a[:-1, :]
    nb[:-1, :] += a[1:, :]
    nb[:, 1:] += a[:, :-1]
    nb[:, :-1] += a[:, 1:]
    t = np.abs(b) + (abs(lam) + 4 / h ** 2) * a + nb / h ** 2
    return np.linalg.norm(r) / bn, 8 * np.finfo(float).eps * np.linalg.norm(t) / bn


def test_batch_fp64_matches_oracle():
    probs = inputs.uneven_problem(**SMALL)
    bt = api.Batch([p[0] for p in probs], [p[1] for p in probs], api.config())
    zs = [torch.empty(lam.size, N, N, dtype=torch.complex128, device="cuda") for N, lam, _ in probs]
    out = bt.solve(zs, [dev(b) for _, _, b in probs])
    torch.cuda.synchronize()
    for (N, lam, b), z, (it, rr) in zip(probs, zs, out):
        om = lfa.omega_table(lam, N, mode="lfa")
        zo, ito, rro = core.shifted_solve_batch(N, lam, om, b, tol=1e-10)
        assert np.array_equal(it, ito), (N, it, ito)
        assert np.all(rr <= 1e-10)
        assert rel_per_vector(z.cpu().numpy(), zo) < 1e-12
    bt.destroy()


@pytest.mark.parametrize("N,n", [(63, 8), (255, 16)])
def test_refined_solve_reaches_fp64_tolerance_graphs_on_and_off(N, n):
    rng = np.random.default_rng(N)
    lam = inputs.random_shifts(rng, n)
    b = inputs.complex_rhs(rng, n, N)
    bd = dev(b)
    zs = {}
    for g in (1, 0):
        s = torch.cuda.Stream()
        # fused_variant 1: no timed choice between implementations, so that both contexts
        # run the same kernels and the answers can be compared bit for bit
        c = api.Context(N, n, lam, cfg=api.config(precision=1, cuda_graphs=g, fused_variant=1),
                        stream=s.cuda_stream)
        z = torch.zeros(n, N, N, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        it, rr = c.shifted_solve_refined(z, bd)
        torch.cuda.synchronize()
        zs[g] = (z.cpu().numpy(), it, rr)
        c.destroy()
    z, it, rr = zs[1]
    assert np.array_equal(z, zs[0][0]) and np.array_equal(it, zs[0][1])
    h = 1.0 / (N + 1)
    mu = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    om = lfa.omega_table(lam, N, mode="lfa")
    zo, _, _ = core.shifted_solve_batch(N, lam, om, b, tol=1e-13, maxit=200)
    for j in range(n):
        rel, noise = oracle_relres(N, lam[j], b[j], z[j])
        assert rel <= 1e-10 and abs(rr[j] - rel) <= 1e-6 * rel + noise
        # (lam + A) is normal with eigenvalues lam + mu_k, |lam + mu_k| >= mu_min + Re lam
        bound = (rel + 1e-13) * np.linalg.norm(b[j]) / (mu + lam[j].real)
        assert np.linalg.norm(z[j] - zo[j]) <= 1.01 * bound


def test_batch_refined_equals_single_contexts():
    probs = inputs.uneven_problem(**SMALL)
    bt = api.Batch([p[0] for p in probs], [p[1] for p in probs],
                   api.config(precision=1, fused_variant=1))
    zs = [torch.empty(lam.size, N, N, dtype=torch.complex128, device="cuda") for N, lam, _ in probs]
    bs = [dev(b) for _, _, b in probs]
    out = bt.solve(zs, bs)
    torch.cuda.synchronize()
    for (N, lam, b), z, bdev, (it, rr) in zip(probs, zs, bs, out):
        c = api.Context(N, lam.size, lam, cfg=api.config(precision=1, cuda_graphs=0, fused_variant=1))
        z1 = torch.empty_like(z)
        it1, rr1 = c.shifted_solve_refined(z1, bdev)
        torch.cuda.synchronize()
        assert np.array_equal(z.cpu().numpy(), z1.cpu().numpy())
        assert np.array_equal(it, it1) and np.array_equal(rr, rr1)
        for j in range(lam.size):
            rel, noise = oracle_relres(N, lam[j], b[j], z.cpu().numpy()[j])
            assert rel <= 1e-10 and abs(rr[j] - rel) <= 1e-6 * rel + noise
        c.destroy()
    bt.destroy()


def test_batch_uneven8_full_size_sampled():
    """The eight-instance workload at full size (775,123,472 unknowns), FP32 multigrid with
    FP64 refinement to 1e-10 per shift, in the launch configuration of a timed run; the
    oracle recomputes the FP64 residual of the first, middle and last shift of every
    instance."""
    w = inputs.WORKLOADS["uneven-8"]
    probs = inputs.uneven_problem(w["Ns"], w["ns"], w["seed"])
    bt = api.Batch([p[0] for p in probs], [p[1] for p in probs], api.config(precision=1))
    zs = [torch.empty(lam.size, N, N, dtype=torch.complex128, device="cuda") for N, lam, _ in probs]
    bs = [dev(b) for _, _, b in probs]
    out = bt.solve(zs, bs)
    torch.cuda.synchronize()
    for (N, lam, b), z, (it, rr) in zip(probs, zs, out):
        assert np.all(rr <= 1e-10)
        n = lam.size
        for j in sorted({0, n // 2, n - 1}):
            zj = z[j].cpu().numpy()
            rel, noise = oracle_relres(N, lam[j], b[j], zj)
            assert rel <= 1e-10 and abs(rr[j] - rel) <= 1e-6 * rel + noise
    bt.destroy()


@pytest.mark.parametrize("graphs", [1, 0])
def test_batched_launches_per_level(graphs):
    """FP32 V(1,1) batches run every cycle of all instances as one launch per multigrid level
    (2 G + 2 launches, G the most global levels of an instance): uneven grids 63 (solved
    inside the coarse kernel), 127, 255, 511 with 4 to 16 shifts, every shift refined to the
    oracle's FP64 relative residual <= 1e-10; graphs on and off give the same answers."""
    probs = inputs.uneven_problem((63, 127, 255, 511), (4, 8, 8, 16), seed=9)
    bt = api.Batch([p[0] for p in probs], [p[1] for p in probs], api.config(precision=1, cuda_graphs=graphs))
    batched, per_cycle, _ = bt.info()
    assert batched and per_cycle == 2 * 3 + 2  # 511: global levels 511, 255, 127
    zs = [torch.empty(lam.size, N, N, dtype=torch.complex128, device="cuda") for N, lam, _ in probs]
    bs = [dev(b) for _, _, b in probs]
    out = bt.solve(zs, bs)
    torch.cuda.synchronize()
    assert bt.info()[2] > 0
    for (N, lam, b), z, (it, rr) in zip(probs, zs, out):
        assert np.all(rr <= 1e-10)
        for j in range(lam.size):
            rel, noise = oracle_relres(N, lam[j], b[j], z.cpu().numpy()[j])
            assert rel <= 1e-10 and abs(rr[j] - rel) <= 1e-6 * rel + noise
    # the same batch once more: identical answers (the graphs or launches replay)
    zs2 = [torch.empty_like(z) for z in zs]
    out2 = bt.solve(zs2, bs)
    torch.cuda.synchronize()
    for z, z2, (it, rr), (it2, rr2) in zip(zs, zs2, out, out2):
        assert torch.equal(z, z2) and np.array_equal(it, it2)
    bt.destroy()
