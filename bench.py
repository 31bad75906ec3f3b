#!/usr/bin/env python
"""Throughput of the ParaDIAG step (alpha-circulant backward Euler, heat equation on the
unit square) on one GB300: shifted solves per second to relative residual 1e-10, for
the FP32-multigrid + FP64-refinement form (the value) and the plain FP64 form (beside
it), with the roofline of the dominant kernel and the FP64 CPU oracle as a baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload paradiag-2047]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

One step = one whole paradiag_solve: transforms, n batched multigrid solves, refinement.
Under torchrun every rank solves its own independent problem (weak scaling, no
collective on the data path); the time is the maximum over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shifted solves/s to rel.res 1e-10: FP32+IR vs FP64 on GB300; % HBM peak"
HBM_FALLBACK_GBS = 6800.0


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def peak_tf32():
    """Dense TF32 tensor peak: the measured sustained bf16 GEMM rate (the transforms run inside
    a long step) times the nominal TF32 / bf16 ratio 1.1 / 2.25; the nominal 1100 TF/s
    without the measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return round(float(d["bf16_tflops_sustained"]) * 1.1 / 2.25, 1)
    except Exception:
        return 1100.0


def traffic_table():
    """Per-launch DRAM bytes from the committed ncu summaries (kernel class -> bytes)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    out = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                p = line.split()
                if len(p) >= 3 and not line.startswith("#"):
                    out[(p[0], p[1])] = float(p[2])
    return out


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        smax = float(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


class OracleSample:
    """Times the FP64 CPU oracle on a bounded sample of the workload and scales it to the
    whole step: the forward transform on `pts` of the m grid points (x m/pts, and x2 for
    the inverse transform of the same size) plus the multigrid solves of `threads` of the n
    shifted systems on the full grid, one per thread (x n/threads).  The inputs, the
    transformed right-hand sides of the sampled shifts and their relaxation table are
    prepared once; every call of time() repeats only the timed oracle work."""

    def __init__(self, workload, threads, f=None, u0=None):
        from oracle import core, lfa
        from paper_2203_11154_gb300 import inputs

        self.core = core
        w = inputs.WORKLOADS[workload]
        self.workload = workload
        N, n, tau, alpha = w["N"], w["n"], w["tau"], w["alpha"]
        self.N, self.n = N, n
        self.s = max(1, min(threads, n))
        core.set_threads(threads)
        if f is None:
            f, u0 = inputs.paradiag_problem(N, n, seed=w["seed"])
        lam, V, Vinv = core.alpha_circulant(n, tau, alpha)
        fhat = core.assemble_rhs(N, n, tau, f, u0).reshape(n, -1)
        self.m = fhat.shape[1]
        self.pts = min(self.m // 16, 65536)
        self.Vinv = Vinv
        self.x = np.ascontiguousarray(fhat[:, :self.pts])
        sel = np.linspace(0, n - 1, self.s).astype(int)
        self.lam = lam[sel]
        self.g = (Vinv[sel] @ fhat).reshape(self.s, N, N)
        del fhat
        self.om = lfa.omega_table(self.lam, N, mode="lfa")

    def time(self):
        """(solves/s of the whole step scaled from the sample, seconds of oracle work, text)."""
        core = self.core
        t0 = time.perf_counter()
        core.time_transform(self.Vinv, self.x)
        t_tr = time.perf_counter() - t0
        t0 = time.perf_counter()
        core.shifted_solve_batch(self.N, self.lam, self.om, self.g, tol=1e-10)
        t_mg = time.perf_counter() - t0
        m, ms, n, s = self.m, self.pts, self.n, self.s
        step = 2 * t_tr * (m / ms) + t_mg * (n / s)
        desc = ("forward transform of %d of %d grid points (x%.0f, x2 for the inverse) and "
                "multigrid solves of %d of %d shifted systems on the full %dx%d grid (x%.1f); "
                "%s workload" % (ms, m, m / ms, s, n, self.N, self.N, n / s, self.workload))
        return n / step, t_tr + t_mg, desc


def rank_seed(workload, rank):
    """Each rank solves its own problem: the workload's input recipe with seed + rank
    (weak scaling; no collective on the data path)."""
    from paper_2203_11154_gb300 import inputs
    return inputs.WORKLOADS[workload]["seed"] + rank


def max_over_ranks(x, world, device):
    """The step time of the job: the maximum over ranks (all_reduce MAX)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n, steps, world, ms):
    """Shifted solves of all ranks per second: n systems per step on each of `world` ranks,
    over the slowest rank's time for `steps` steps."""
    return n * steps * world / (ms / 1e3)


def bench_config(workload):
    """The workload description both arms print."""
    from paper_2203_11154_gb300 import inputs
    w = inputs.WORKLOADS[workload]
    f_mb = (w["n"] * w["N"] * w["N"] * 8) >> 20
    return {"workload": workload, "N": w["N"], "n": w["n"], "tau": w["tau"], "alpha": w["alpha"],
            "cycle": "V(1,1)", "smoother": "additive element-wise Vanka",
            "omega": "LFA per shift and level", "tol_allatonce": 1e-10,
            "precision": "FP32 multigrid + FP64 refinement on eq. (1)",
            "l2": "inputs larger than L2 (f: %d MB)" % f_mb,
            "imag_check": "max |Im((V kron I) z)| formed in every inverse transform",
            "parallelism": "one independent problem per rank"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    vals, secs = [], []
    sample = OracleSample(args.workload, cores)
    for k in range(args.warmup + args.steps):
        v, sec, desc = sample.time()
        if k >= args.warmup:
            vals.append(v)
            secs.append(sec)
    v = float(np.median(vals))
    from paper_2203_11154_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * w["n"] / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.workload),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": "solves/s",
                             "sample": desc, "sample_seconds_median": float(np.median(secs))},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_batch(args, rank, world, barrier, rank_max, local):
    """The batched uneven form: eight independent shifted-system problems of different
    sizes (528 systems) solved together by pd_batch, FP32 multigrid with FP64 refinement of
    every system to relative residual 1e-10.  A step = one pd_batch_solve of all instances
    (inputs resident on the device).  Returns (solves/s, the line's other keys)."""
    import torch
    from paper_2203_11154_gb300 import api, inputs
    w = inputs.WORKLOADS["uneven-8"]
    probs = inputs.uneven_problem(w["Ns"], w["ns"], w["seed"] + rank)
    bt = api.Batch([p[0] for p in probs], [p[1] for p in probs], api.config(precision=1))
    bs = [torch.from_numpy(p[2]).cuda() for p in probs]
    zs = [torch.empty_like(b) for b in bs]
    total = sum(p[1].size for p in probs)
    for _ in range(args.warmup):
        out = bt.solve(zs, bs)
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = Clocks(local)
    clocks.start()
    l0 = bt.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out = bt.solve(zs, bs)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    launches = bt.launch_count() - l0
    ms = rank_max(e0.elapsed_time(e1))
    batched, per_cycle, _ = bt.info()
    rr = max(float(np.max(r)) for _, r in out)
    cyc = max(int(np.max(it)) for it, _ in out)
    value = job_throughput(total, args.steps, world, ms)
    keys = {"ms_per_step": ms / args.steps,
            "config": {"workload": "uneven-8", "N": list(w["Ns"]), "n": list(w["ns"]),
                       "systems": total, "precision": "FP32 multigrid + FP64 refinement per system",
                       "l2": "inputs larger than L2 (RHS: %d MB)" % (sum(b.numel() for b in bs) * 16 >> 20)},
            "launches_per_cycle": per_cycle if batched else None,
            "relres_shift_max": rr, "fp32_cycles_max": cyc, "clocks": ck,
            "gpu_launches": launches}
    bt.destroy()
    del bs, zs
    return value, keys


def run_batch(args, rank, world, barrier, rank_max, local):
    value, keys = measure_batch(args, rank, world, barrier, rank_max, local)
    line = {"metric": "shifted solves/s to rel.res 1e-10 (batched uneven instances)",
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "e2e": None}
    line.update(keys)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def examples_shifts():
    """The shifted systems of Sec. 3's examples: Example 1 (the BVM B of eq. (9), n = 256,
    h = tau = 1/256), Example 2 (the quasi-BVM B of eq. (10), n = 256 plus the extra step,
    beta = 0.01, h = tau = 1/256) and Example 3 (Helmholtz shifts -j^2 (1 - 0.5 i),
    j h <= 1/2, h = 1/128).  The library diagonalises the B matrices."""
    from paper_2203_11154_gb300 import api, inputs
    n = 256
    return [("example1", 255, api.pd_diagonalize(inputs.bvm_time_matrix(n))[0]),
            ("example2", 255, api.pd_diagonalize(inputs.quasi_bvm_time_matrix(n, 0.01))[0]),
            ("example3", 127, inputs.helmholtz_shifts(1.0 / 128))]


def run_examples(args):
    """Sec. 3's setting (W(1,0) cycles, coarsest h0 = 1/8, fixed omega, relative residual
    1e-8, FP64) on the shifts of Examples 1-3 with seeded complex U(-1,1) right-hand sides:
    the cycle count of every shift for the Vanka smoother (omega = 24/25) and damped Jacobi
    (omega = 4/5), and the GPU-timed solves/s of both (the paper reports Vanka about three
    times faster in serial MATLAB).  Shifts are solved 128 at a time (one context each)."""
    import torch
    from paper_2203_11154_gb300 import api, inputs
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream()
    out = {"metric": "cycle counts and solves/s, Vanka vs damped Jacobi (Sec. 3 examples)",
           "cycle": "W(1,0), coarsest 7x7 (h0 = 1/8), fixed omega, tol 1e-8, FP64", "examples": {}}
    for name, N, lam in examples_shifts():
        rng = np.random.default_rng(11)
        b = inputs.complex_rhs(rng, lam.size, N)
        ex = {"N": N, "n": int(lam.size)}
        for sm, sname in ((0, "vanka"), (1, "jacobi")):
            cfg = api.config(cycle_gamma=2, nu1=1, nu2=0, coarsest_n=7, omega_mode=0, tol=1e-8,
                             maxit=1000, precision=0, smoother=sm)
            chunks = []
            for a in range(0, lam.size, 128):
                sl = slice(a, min(a + 128, lam.size))
                c = api.Context(N, lam[sl].size, lam[sl], cfg=cfg)
                bd = torch.from_numpy(np.ascontiguousarray(b[sl])).cuda()
                chunks.append((c, bd, torch.empty_like(bd)))
            its = []
            for c, bd, z in chunks:  # warm-up and the counts
                it, _ = c.shifted_solve_batched(z, bd, raise_on_noconv=False)
                its.append(it)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                for c, bd, z in chunks:
                    c.shifted_solve_batched(z, bd, raise_on_noconv=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            it = np.concatenate(its)
            ex[sname] = {"cycles": it.tolist(), "cycles_min": int(it.min()), "cycles_max": int(it.max()),
                         "cycles_mean": float(it.mean()), "ms_per_solve_of_all_shifts": ms,
                         "solves_per_s": lam.size / (ms * 1e-3)}
            for c, _, _ in chunks:
                c.destroy()
        ex["vanka_speedup_vs_jacobi"] = ex["vanka"]["solves_per_s"] / ex["jacobi"]["solves_per_s"]
        out["examples"][name] = ex
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="paradiag-2047",
                    choices=["paradiag-511", "paradiag-511-128", "paradiag-1023", "paradiag-2047", "uneven-8",
                             "examples"])
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 form beside the value (default: the smaller "
                         "of --steps and 3 at N = 2047, else --steps)")
    ap.add_argument("--transforms", default="fft", choices=["fft", "tc"],
                    help="route of the time transforms: the Gamma-weighted FFTs of the "
                         "alpha-circulant V, or V and V^{-1} as dense TF32x3 tcgen05 products "
                         "(the route of a general B)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-uneven8", action="store_true",
                    help="leave out the batched uneven-instances figure of the default line")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "examples":
        return run_examples(args)

    import torch
    import torch.distributed as dist

    from paper_2203_11154_gb300 import api, inputs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # a stream of its own (not the legacy default stream), so that the library can replay
    # its multigrid cycles as CUDA graphs
    torch.cuda.set_stream(torch.cuda.Stream())

    def barrier():
        if world > 1:
            dist.barrier()

    def rank_max(x):
        return max_over_ranks(x, world, "cuda")

    if args.workload == "uneven-8":
        return run_batch(args, rank, world, barrier, rank_max, local)

    w = inputs.WORKLOADS[args.workload]
    N, n, tau, alpha = w["N"], w["n"], w["tau"], w["alpha"]
    f, u0 = inputs.paradiag_problem(N, n, seed=rank_seed(args.workload, rank))
    fd = torch.from_numpy(f).cuda()
    u0d = torch.from_numpy(u0).cuda()
    u = torch.empty_like(fd)
    stream = torch.cuda.current_stream()

    def timed(ctx, steps, warmup, profile=False, clocks=None):
        out = None
        for _ in range(warmup):
            out = ctx.paradiag_solve(u, fd, u0d)
        barrier()
        torch.cuda.synchronize()
        if profile:
            ctx.profile_enable(True)
        l0 = ctx.launch_count()
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")  # profiler captures filter on this range
        e0.record(stream)
        for _ in range(steps):
            out = ctx.paradiag_solve(u, fd, u0d)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        barrier()
        ck = clocks.stop() if clocks else None
        ms = rank_max(e0.elapsed_time(e1))
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile_enable(False)
        return ms, out, prof, ctx.launch_count() - l0, ck

    # FP32 multigrid inside FP64 refinement (the value)
    ctx = api.alpha_circulant_context(N, n, tau, alpha, precision=1, imag_check=1,
                                      fft_transforms=int(args.transforms == "fft"))
    clocks = Clocks(local)
    ms_ir, out_ir, _, launches, ck = timed(ctx, args.steps, args.warmup, clocks=clocks)
    value = job_throughput(n, args.steps, world, ms_ir)
    # per-kernel durations: CUDA events around every launch, in a second pass of the same
    # K steps (kept out of the timed pass above, whose step time they would inflate)
    ms_prof, _, prof, _, _ = timed(ctx, args.steps, 0, profile=True)
    # the fused smoothing kernels the set-up autotuner chose per level (1 TMA tiles, 2 warp
    # streams with rows per segment, 0 none)
    autotune = [{"level": l, "variant": v, "rows_per_segment": sg} for l, (v, sg) in enumerate(ctx.fused_choices())]

    # end to end through the host-buffer C ABI call (pinned host memory; every step copies
    # its f and u0 in and its u out inside the timed region, the copies of neighbouring
    # steps overlapping the solves through paradiag_solve_host_batch)
    e2e = None
    if not args.no_e2e:
        fh = torch.from_numpy(f).pin_memory()
        u0h = torch.from_numpy(u0).pin_memory()
        uhs = [torch.empty_like(fh).pin_memory() for _ in range(2)]

        def host_steps(k):
            return ctx.paradiag_solve_host_batch([uhs[j % 2] for j in range(k)], [fh] * k, [u0h] * k)

        host_steps(max(1, args.warmup))
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = host_steps(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e2e = rank_max(e0.elapsed_time(e1))
        e2e = {"value": job_throughput(n, args.steps, world, ms_e2e), "unit": "solves/s",
               "h2d_bytes_per_step": int(fh.numel() * 8 + u0h.numel() * 8),
               "d2h_bytes_per_step": int(uhs[0].numel() * 8), "ms_per_step": ms_e2e / args.steps,
               "relres_allatonce_max": max(o["relres_allatonce"] for o in outs),
               "api": "paradiag_solve_host_batch (copies of step k+1 in and k-1 out during step k)"}
        del fh, u0h, uhs
    ctx.destroy()

    # plain FP64 (beside the value)
    ctx64 = api.alpha_circulant_context(N, n, tau, alpha, precision=0, imag_check=1,
                                        fft_transforms=int(args.transforms == "fft"))
    k64 = args.fp64_steps or (min(args.steps, 3) if N >= 2047 else args.steps)
    ms64, out64, _, _, _ = timed(ctx64, k64, max(3, min(args.warmup, 3)))
    ctx64.destroy()
    value64 = job_throughput(n, k64, world, ms64)

    # the batched uneven-instances form (eq. (2) for eight grids at once), its own timed
    # region after this one
    uneven8 = None
    if not args.no_uneven8 and args.workload == "paradiag-2047":
        uv, uk = measure_batch(args, rank, world, barrier, rank_max, local)
        uneven8 = {"value": uv, "unit": "solves/s", "steps": args.steps}
        uneven8.update(uk)

    # roofline of the dominant kernel class (its own launch times, live in the timed region)
    peak, peak_src = measured_peaks()
    total = sum(v[0] for v in prof.values())
    kernels = []
    for name, (kms, nl, by) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
        if nl == 0:
            continue
        kernels.append({"kernel": name, "launches": nl, "ms": round(kms, 3),
                        "share": round(kms / total, 4),
                        "gbs": round(by / (kms * 1e-3) / 1e9, 1) if kms > 0 else None})
    top = kernels[0]
    tname = top["kernel"]
    tms, tn, tby = prof[tname]
    achieved = tby / (tms * 1e-3) / 1e9
    traffic = traffic_table().get((args.workload, tname))
    roofline = {"bound": "hbm", "kernel": tname, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": traffic, "alg_bytes_per_launch": tby / tn,
                "avg_launch_us": 1e3 * tms / tn}

    # the whole solve against the HBM peak: algorithmic bytes of every kernel of a step
    # (from the profiled pass) over the step time of the timed pass
    step_bytes = sum(v[2] for v in prof.values()) / args.steps
    solve_gbs = step_bytes / (ms_ir / args.steps * 1e-3) / 1e9
    solve_hbm = {"alg_bytes_per_step": step_bytes, "achieved": round(solve_gbs, 1), "peak": peak,
                 "unit": "GB/s", "frac": round(solve_gbs / peak, 4)}

    # the time transforms against both of their bounds: HBM (bytes per launch as profiled)
    # and the TF32 tensor pipe (TF32x3: three real products per complex-by-real product)
    transforms = {"route": args.transforms}
    for name in ("forward", "inverse"):
        if name not in prof or prof[name][1] == 0:
            continue
        kms, nl, by = prof[name]
        t = {"launches": nl, "avg_launch_us": round(1e3 * kms / nl, 1),
             "gbs": round(by / (kms * 1e-3) / 1e9, 1), "frac_hbm": round(by / (kms * 1e-3) / 1e9 / peak, 4)}
        if args.transforms == "tc":
            # Re and Im rows of W (n x n) times the n x N^2 real (or Re-of-complex) operand,
            # each a sum of three TF32 products
            flops = 3 * 2 * (2 * n) * n * N * N * nl
            tf32_peak = peak_tf32()
            t["tflops_issued"] = round(flops / (kms * 1e-3) / 1e12, 1)
            t["tf32_peak"] = tf32_peak
            t["frac_tensor"] = round(flops / (kms * 1e-3) / 1e12 / tf32_peak, 4)
        transforms[name] = t

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_ir / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": dict(bench_config(args.workload), time_transforms=args.transforms),
            "launch": "multigrid cycles replayed as CUDA graphs on a non-default stream",
            "relres_allatonce": out_ir["relres_allatonce"],
            "refine_steps": out_ir["refine_steps"], "cycles_max": out_ir["cycles_max"],
            "imag_max": out_ir["imag_max"],
            "fp64": {"value": value64, "unit": "solves/s", "ms_per_step": ms64 / k64,
                     "steps": k64, "relres_shift_max": out64["relres_shift_max"],
                     "relres_allatonce": out64["relres_allatonce"],
                     "cycles_max": out64["cycles_max"]},
            "speedup_vs_fp64": value / value64, "uneven8": uneven8, "autotune": autotune,
            "clocks": ck, "e2e": e2e, "gpu_launches": launches,
            "roofline": roofline, "solve_hbm": solve_hbm, "transforms": transforms,
            "kernels": kernels,
            "kernel_timing": "CUDA events around each launch on the context's stream, in a "
                             "second pass of the same %d steps (%.2f ms/step with the events)"
                             % (args.steps, ms_prof / args.steps)}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the sample repeated until about 10 s of oracle work (at most 16 times); the median
        cores = os.cpu_count() or 1
        vals, tot = [], 0.0
        sample = OracleSample(args.workload, cores, f, u0)
        while tot < 10.0 and len(vals) < 16:
            v, sec, desc = sample.time()
            vals.append(v)
            tot += sec
        line["cpu_baseline"] = {"value": float(np.median(vals)), "unit": "solves/s", "cores": cores,
                                "kind": "oracle", "sample": desc + "; median of %d repetitions" % len(vals),
                                "sample_seconds": round(tot, 2)}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
