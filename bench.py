#!/usr/bin/env python
"""Throughput of the VMC hot path on one GB300: Pfaffian hop-updates/s.

One step = every walker samples `--samples` measurements (one sweep of Ne
proposals before each, then E_loc and the O_k row), followed by one SR step
(dense S, Cholesky) and the rebuild of every walker's inverse for the new
parameters.  Workload: 16x16 Hubbard, U/t = 8, Ne = 224 (n = 0.875),
anti-periodic in x and y, Gutzwiller + distance Jastrow + 2x2-sublattice
pair orbitals (Np = 1069), 4096 walkers, synthetic seeded inputs.

The headline `value` is the mixed form (FP32 sweep, FP64 from-scratch
inverses, FP64 energies and solve); the plain FP64 form runs the same steps
and is reported beside it, with the energy difference of the two forms on
identical configurations.  After the timed steps, the pair correlations of
the measurement mode (vmc_measure_corr) are timed on the mixed context's
configurations and reported in their own object.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# FP32 lanes and FP64 FMA units per SM, SM count and maximum clock of GB300
# (sm_103): the ALU peaks the sweep (FP32) and the from-scratch inverses
# (FP64) are judged against.
SMS, FP32_LANES, FP64_UNITS, SM_MAX_MHZ = 152, 128, 2, 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = SMS * FP64_UNITS * 2 * SM_MAX_MHZ * 1e6 / 1e12
# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernels at 4096 walkers (profiles/k_sample_float_hubbard16x16_w4096.md,
# profiles/k_init_float_hubbard16x16_w4096.md); proportional to walkers.
TRAFFIC_SWEEP_4096 = 225.731328e6 + 181.081344e6
TRAFFIC_INIT_4096 = 6.181120e6 + 160.923392e6
# k_corr<float> (pair correlations), DRAM read + write per launch at 4096
# walkers (profiles/k_corr_float_hubbard16x16_w4096.md).
TRAFFIC_CORR_4096 = 229.7047e6


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--walkers", type=int, default=4096)
    ap.add_argument("--samples", type=int, default=4)
    ap.add_argument("--recompute", type=int, default=256)
    ap.add_argument("--equil", type=int, default=10)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-corr", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def workload():
    from paper_1711_11418_gb300 import inputs
    return inputs.square16_hubbard()


METRIC = "Pfaffian hop-updates/s, 16x16 Hubbard (mixed/batched form; plain FP64 beside)"


def workload_config(args, prob, world):
    """The `config` object of both arms: the workload, with its sizes."""
    return {"workload": "hubbard_16x16_U8_Ne224_apbc", "walkers": args.walkers,
            "samples_per_walker_per_step": args.samples, "sweeps_between_samples": 1,
            "proposals_per_sweep": prob.Ne, "p_exchange": prob.p_exchange, "Np": prob.Np,
            "recompute_every_accepted": args.recompute,
            "sr": "dense S (FP64 SYRK plain / split-BF16 tensor cores mixed); FP64 Cholesky "
                  "plain, FP64 iterative refinement on an FP32 inverse mixed; shift_rel 1e-3, "
                  "dtau 0.05",
            "l2": "no flush: walker state (4096 x 50.6 KB FP32 inverses) exceeds the 129 MB L2",
            "parallelism": "replicas" if world > 1 else "single"}


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def reduce_over_ranks(torch, value, op):
    """`value` reduced over all ranks ("max" or "sum"); the value itself when
    no process group is running.  Replicas are timed by the slowest rank and
    credited with the work of all."""
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()):
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline and reference arm: the oracle, as it stands
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    wid, n_props, seconds = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    from paper_1711_11418_gb300 import inputs
    from oracle.sampler import Chain
    from oracle.wavefunction import Wavefunction
    p = inputs.square16_hubbard()
    wf = Wavefunction(p)
    ele = inputs.initial_configs(p.Ns, p.Ne, 1, False, 5000 + wid)[0]
    ch = Chain(wf, ele, seed=1, system=0, walker=wid, p_exchange=p.p_exchange)
    t0 = time.perf_counter()
    k = 0
    while (n_props and k < n_props) or (not n_props and time.perf_counter() - t0 < seconds):
        ch.propose()
        k += 1
    return k, time.perf_counter() - t0


def oracle_pool(cores):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return mp.get_context("spawn").Pool(cores)


def cpu_baseline(pool, cores, seconds):
    t0 = time.perf_counter()
    res = pool.map(_oracle_worker, [(w, 0, seconds) for w in range(cores)])
    wall = time.perf_counter() - t0
    props = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    return {"value": props / t, "unit": "proposals/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent chains (one per core) of the 16x16 Hubbard "
                      f"workload, {props} proposals in {t:.1f} s, each ratio from two "
                      f"Parlett-Reid Pfaffians; measurement and SR not included",
            "wall_s": round(wall, 2)}


def run_reference(args):
    rank, _, world = dist_info()
    if rank != 0:
        return
    cores = min(os.cpu_count() or 1, 64)
    pool = oracle_pool(cores)
    # calibrate: proposals per core per step so that a step takes ~2 s
    k, t = pool.map(_oracle_worker, [(0, 20, 0)])[0]
    per = max(4, int(2.0 * k / max(t, 1e-6)))
    times, props = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(w, per, 0) for w in range(cores)])
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            props.append(sum(r[0] for r in res))
    pool.close()
    value = sum(props) / sum(times)
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "proposals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args, workload(), 1),
            "cpu_baseline": {"value": value, "unit": "proposals/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: {cores} chains of the workload (one per core) "
                                       f"x {per} proposals, ratios from two Parlett-Reid "
                                       f"Pfaffians; measurement and SR not included"},
            "e2e": {"value": value, "unit": "proposals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def measured_alu_peaks(torch):
    """FP64 and FP32 (non-tensor) GEMM throughput of this GPU, TFLOP/s: the
    ALU ceilings the sweep kernels are judged against (library GEMM, best of 5)."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n in (("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192)):
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            torch.matmul(a, b)
            best = 0.0
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
            out[name] = best
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def flops_of(d, N, precision):
    """Algorithmic FLOPs of the sweep kernel from its counters: a tested hop
    2N (one dot product), a tested exchange 2N^2 + 6N (a row-vector times
    M^-1 and the 2x2 entries), an accepted hop 4N^2 (that product and the
    rank-1 update), an accepted exchange 6N^2 (rank-2 update), a measured hop
    ratio 2N, a measured exchange ratio 2N^2 + 6N.  Returns (flops in the
    sweep's arithmetic type, FP64 in-sweep recompute flops 2N^3 each)."""
    main = (2 * N * d["n_hop_tested"] + (2 * N * N + 6 * N) * d["n_exchange_tested"]
            + 4 * N * N * d["n_hop_accepted"] + 6 * N * N * d["n_exchange_accepted"]
            + 2 * N * d["n_measured_hops"] + (2 * N * N + 6 * N) * d["n_measured_exchanges"])
    rec = 2 * N ** 3 * d["n_recomputes"]
    return main, rec


def delta(a, b):
    return {k: b[k] - a[k] for k in b if isinstance(b[k], int)}


def run_arm(vmc, prob, args, precision, stream, torch, world):
    W, S = args.walkers, args.samples
    ctx = vmc.Context(prob, W, seed=1234 + int(os.environ.get("RANK", 0)), precision=precision,
                      max_samples=S, recompute_every=args.recompute if precision == vmc.MIXED else -1,
                      stream=stream.cuda_stream)
    ctx.sample(args.equil, 0, 0)                        # equilibration (untimed)
    delay = None
    if precision == vmc.MIXED:
        # delayed-update depth by the autotuner, timed on the step's launch
        # shape (one sweep and one measurement; these are warm-up sweeps)
        delay, delay_ms = ctx.tune_delay(sweeps=1, candidates=(1, 2, 4, 8))
        delay = {"chosen": delay, "ms_per_sweep": delay_ms}
    # plain form: FP64 Cholesky; mixed form: FP64 iterative refinement on an
    # FP32 inverse (FP64 Cholesky if it does not reach the residual target)
    sr = dict(dtau=0.05, shift_rel=1e-3, shift_abs=0.0,
              solver=vmc.MIXED_IR if precision == vmc.MIXED else vmc.CHOLESKY, cg_eps=1e-12)
    reps = []

    def step():
        ctx.sample(0, S, 1)
        reps.append(ctx.sr_step(**sr))

    for _ in range(args.warmup):
        step()
    ctx.enable_timing(True)
    ctx.kernel_times()
    st0 = ctx.measure()
    l0 = ctx.kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    energies = []
    for _ in range(args.steps):
        step()
        energies.append(ctx.measure()["energy"])
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = reduce_over_ranks(torch, e0.elapsed_time(e1), "max")
    st1 = ctx.measure()
    kt = ctx.kernel_times()
    launches = ctx.kernel_launches() - l0
    d = delta(st0, st1)
    props_all = reduce_over_ranks(torch, d["n_proposals"], "sum")
    timed = reps[-args.steps:]
    solve = dict(solver="mixed_ir" if precision == vmc.MIXED else "cholesky_fp64",
                 refinement_steps_max=max(r["cg_iters"] for r in timed),
                 fallbacks=sum(r["fallback"] for r in timed),
                 rel_residual_max=max(r["rel_residual"] for r in timed))
    return ctx, dict(ms=ms, stats=d, kt=kt, launches=launches, clocks=clk,
                     energy=statistics.fmean(energies), last=st1, solve=solve,
                     props_all=props_all, sr=sr, delay=delay)


def run_ours(args):
    rank, local, world = dist_info()
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    pool = None
    cores = min(os.cpu_count() or 1, 64)
    if rank == 0 and world == 1 and not args.no_cpu:
        pool = oracle_pool(cores)             # spawn before the first CUDA call
    from paper_1711_11418_gb300 import build, vmc
    build.build()
    prob = workload()
    N = prob.N
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx, mixed = run_arm(vmc, prob, args, vmc.MIXED, stream, torch, world)
        fp64 = None
        if not args.no_fp64:
            ctx64, fp64 = run_arm(vmc, prob, args, vmc.FP64, stream, torch, world)
            ctx64.close()
        # Energy accuracy of the mixed form on identical configurations
        ele, ctr = ctx.get_configs()
        params = ctx.get_params()
        check = vmc.Context(prob.copy_with(params=params), args.walkers, seed=1, precision=vmc.FP64,
                            max_samples=1, stream=stream.cuda_stream)
        check.set_configs(ele)
        check.sample(0, 1, 0)
        e64 = check.get_samples()[0]
        ctx.sample(0, 1, 0)
        e32 = ctx.get_samples()[0]
        check.close()
        dE = abs(e32.mean() - e64.mean()) / prob.Ns
        dw = abs(e32 - e64) / prob.Ns
        dE_max = float(dw.max())
        dE_p99 = float(sorted(dw)[int(0.99 * (len(dw) - 1))])
        n_over = int((dw > 1e-4).sum())
        # End to end: parameters from pinned host memory, energy and parameters back
        e2e = None
        if not args.no_e2e:
            hp = torch.empty(prob.Np, dtype=torch.float64, pin_memory=True).numpy()
            hp[:] = params
            t0 = time.perf_counter()
            p0 = ctx.measure()["n_proposals"]
            for _ in range(args.steps):
                ctx.set_params(hp)
                ctx.sample(0, args.samples, 1)
                ctx.sr_step(**mixed["sr"])
                hp[:] = ctx.get_params()
                _ = ctx.measure()["energy"]
            torch.cuda.synchronize()
            dt = reduce_over_ranks(torch, time.perf_counter() - t0, "max")
            props = reduce_over_ranks(torch, ctx.measure()["n_proposals"] - p0, "sum")
            e2e = {"value": props / dt, "unit": "proposals/s",
                   "h2d_bytes_per_step": 8 * prob.Np,
                   "d2h_bytes_per_step": 8 * prob.Np + 8 * args.walkers * args.samples + 64}
        # Pair correlations of the walkers' configurations (measurement mode;
        # not part of the optimisation step timed above): device time of the
        # whole measurement and of its ratio kernel, CUDA events on the stream.
        corr = None
        if not args.no_corr:
            ctx.measure_corr()                      # scratch allocation
            runs = [ctx.measure_corr(timing=True)[1] for _ in range(5)]
            k_ms = statistics.median(r[0] for r in runs)
            all_ms = statistics.median(r[1] for r in runs)
            corr = {"k_ms": k_ms, "all_ms": all_ms}
        ctx.close()

    def summarize(r):
        d = r["stats"]
        secs = r["ms"] * 1e-3
        sweep_ms, sweep_n = r["kt"]["sweep"]
        return {"proposals_per_s": r["props_all"] / secs, "ms_per_step": r["ms"] / args.steps,
                "sweep_kernel_ms_per_launch": sweep_ms / max(sweep_n, 1), "sweep_launches": sweep_n,
                "init_ms_per_step": r["kt"]["init"][0] / args.steps,
                "sr_ms_per_step": r["kt"]["sr"][0] / args.steps,
                "acceptance": d["n_accepted"] / max(d["n_proposals"], 1),
                "energy_per_site": r["energy"] / prob.Ns, "recomputes": d["n_recomputes"],
                "sr_solve": r["solve"], "delay_tuner": r["delay"]}

    peaks = measured_alu_peaks(torch)
    sm = summarize(mixed)
    # Rooflines of the two large kernels of the mixed step; the one with more
    # device time in the timed region is reported as `roofline`.
    #  sweep + measurement (k_sample<float>): FP32 FLOPs from its counters per
    #    launch / launch time, against the FP32 ALU peak; its HBM fraction beside;
    #  from-scratch inverses (k_init<float>): 2 N^3 FP64 FLOPs per inverse
    #    (every walker after each SR step, plus in-sweep recomputes) / time,
    #    against the FP64 peak.
    hbm, hbm_src = hbm_peak_gbs()
    scale = args.walkers / 4096.0
    f32, f64rec = flops_of(mixed["stats"], N, "mixed")
    sweep_ms, sweep_n = mixed["kt"]["sweep"]
    t_launch = sweep_ms * 1e-3 / max(sweep_n, 1)
    ach = f32 / max(sweep_n, 1) / t_launch / 1e12
    sweep_gbs = TRAFFIC_SWEEP_4096 * scale / t_launch / 1e9
    roof_sweep = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": ach / FP32_PEAK_TFLOPS, "traffic": TRAFFIC_SWEEP_4096 * scale,
                  "kernel": "k_sample<float> (sweep + measurement)",
                  "ms_in_timed_region": sweep_ms,
                  "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                  "hbm": {"achieved_gbs": sweep_gbs, "peak_gbs": hbm, "frac": sweep_gbs / hbm,
                          "peak_source": hbm_src}}
    init_ms, _ = mixed["kt"]["init"]
    n_inv = args.steps * args.walkers + mixed["stats"]["n_recomputes"]
    ach_init = 2.0 * N ** 3 * n_inv / max(init_ms * 1e-3, 1e-12) / 1e12
    roof_init = {"bound": "alu", "achieved": ach_init, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                 "frac": ach_init / FP64_PEAK_TFLOPS, "traffic": TRAFFIC_INIT_4096 * scale,
                 "kernel": "k_init<float> (FP64 from-scratch inverses)",
                 "ms_in_timed_region": init_ms,
                 "peak_source": "derived: 152 SMs x 2 FP64 FMA units x 2 x 2070 MHz "
                                "(a DFMA throughput loop measured 1.198 TFLOP/s)"}
    roof, roof2 = (roof_init, roof_sweep) if init_ms > sweep_ms else (roof_sweep, roof_init)
    roof["measured_gemm_tflops"] = peaks
    pair_corr = None
    if corr is not None:
        # k_corr<float>: per configuration G_up (Ns N^2 FMA) and, for each of
        # the N sites holding a down electron, G_dn and T (2 N Ns FMA each)
        fl = 2.0 * 3 * prob.Ns * N * N * args.walkers
        ach_c = fl / (corr["k_ms"] * 1e-3) / 1e12
        pair_corr = {
            "what": "all 6 x Ns^2 pair correlations (c+c up/dn, n n, SzSz, S+S-, S.S) of the "
                    f"{args.walkers} walkers' current configurations, mixed form",
            "ms_per_measurement": corr["all_ms"],
            "configurations_per_s": args.walkers / (corr["all_ms"] * 1e-3),
            "roofline": {"bound": "alu", "achieved": ach_c, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach_c / FP32_PEAK_TFLOPS,
                         "traffic": TRAFFIC_CORR_4096 * scale,
                         "kernel": "k_corr<float>", "ms_per_launch": corr["k_ms"],
                         "flops_per_launch": fl,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}}
    line = {
        "metric": METRIC,
        "value": sm["proposals_per_s"], "unit": "proposals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sm["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config(args, prob, world),
        "mixed": sm,
        "plain_fp64": summarize(fp64) if fp64 else None,
        "speedup_mixed_over_fp64": (sm["proposals_per_s"] / summarize(fp64)["proposals_per_s"]) if fp64 else None,
        "energy_check": {"same_configs_dE_per_site_mean": dE, "same_configs_dE_per_site_max": dE_max,
                         "same_configs_dE_per_site_p99": dE_p99,
                         "walkers_over_tolerance": n_over, "walkers": args.walkers,
                         "tolerance": 1e-4,
                         "tolerance_applies_to": "the energy estimate (walker mean)"},
        "roofline": roof,
        "roofline_second": roof2,
        "pair_correlations": pair_corr,
        "clocks": mixed["clocks"],
        "gpu_launches": mixed["launches"],
        "e2e": e2e,
    }
    if pool is not None:
        line["cpu_baseline"] = cpu_baseline(pool, cores, args.cpu_seconds)
        pool.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
