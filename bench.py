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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# FP32 lanes and FP64 FMA units per SM, SM count and maximum clock of GB300
# (sm_103): the ALU peaks the sweep (FP32) and the from-scratch inverses
# (FP64) are judged against.
SMS, FP32_LANES, FP64_UNITS, SM_MAX_MHZ = 152, 128, 2, 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = SMS * FP64_UNITS * 2 * SM_MAX_MHZ * 1e6 / 1e12
# DRAM bytes (read + write) per launch from one ncu capture (one-pass
# metrics) of the current kernels at 4096 walkers
# (profiles/dram_k_sample_k_init_hubbard16x16_w4096.md): a sweep-only launch
# of k_sample<float> and the full rebuild launch of k_init<float>.
TRAFFIC_SWEEP_ONLY_4096 = 434.15e6 + 368.07e6
TRAFFIC_INIT_4096 = 5.54e6 + 366.87e6
# k_corr<float> (pair correlations), DRAM read + write per launch at 4096
# walkers (profiles/k_corr_float_hubbard16x16_w4096.md).
TRAFFIC_CORR_4096 = 230.7e6


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
    ap.add_argument("--recompute", type=int, default=64)
    ap.add_argument("--equil", type=int, default=10)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-df-rebuild", action="store_true",
                    help="skip the mixed form with the opt-in double-float rebuild")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-corr", action="store_true")
    ap.add_argument("--no-others", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--stat-samples", type=int, default=16)
    ap.add_argument("--learned", action="store_true",
                    help="train the plain and the Pfaffian x MLP state at the learned-part "
                         "size and print their energies (one JSON line) instead of the bench")
    ap.add_argument("--learned-steps", type=int, default=60)
    ap.add_argument("--learned-eval", type=int, default=6)
    ap.add_argument("--learned-finetune", type=int, default=40,
                    help="warm-start protocol: SR steps after the plain state's training")
    ap.add_argument("--sweep-only", type=int, default=8)
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


def _oracle_config_worker(args):
    """Oracle proposal and measurement rates on one configured workload (one
    chain per core): `seconds` of proposals, then `n_meas` measurements."""
    name, wid, seconds, n_meas = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    from paper_1711_11418_gb300 import inputs
    from oracle import fock
    from oracle.hamiltonian import local_energy
    from oracle.sampler import Chain
    from oracle.wavefunction import Wavefunction
    p = inputs.ring8_hubbard() if name == "ring8" else inputs.square8_hubbard()
    wf = Wavefunction(p)
    ele = inputs.initial_configs(p.Ns, p.Ne, 1, False, 7000 + wid)[0]
    ch = Chain(wf, ele, seed=1, system=0, walker=wid, p_exchange=p.p_exchange)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < seconds:
        ch.propose()
        k += 1
    t1 = time.perf_counter()
    for _ in range(n_meas):
        n = fock.from_labels(ch.ele, p.Ns)
        local_energy(wf, n)
        wf.log_derivatives(n)
    return k, t1 - t0, n_meas, time.perf_counter() - t1


def cpu_baseline_configs(pool, cores, seconds=4.0):
    """The oracle on the 8-site ring (C1: 64 walkers x 200 samples x 10 sweeps
    per SR step) and the 8x8 lattice (C2: 1024 walkers x 4 samples x 1 sweep):
    proposal and measurement rates on all cores from a bounded sample, and
    the seconds one SR step's sampling would take at those rates (SR solve
    not included: N_p = 19 and 271)."""
    out = {}
    for name, W, S, sweeps, Ne, n_meas in (("ring8", 64, 200, 10, 8, 20),
                                            ("square8", 1024, 4, 1, 64, 2)):
        res = pool.map(_oracle_config_worker, [(name, w, seconds, n_meas) for w in range(cores)])
        pr = sum(r[0] for r in res) / max(r[1] for r in res)
        mr = sum(r[2] for r in res) / max(r[3] for r in res)
        props = W * S * sweeps * Ne
        out[name] = {"proposals_per_s": pr, "measurements_per_s": mr, "cores": cores,
                     "seconds_per_sr_step_est": props / pr + W * S / mr,
                     "sample": f"{cores} chains x {seconds:.0f} s of proposals, then "
                               f"{n_meas} measurements each (E_loc and O_k by Pfaffians); "
                               f"the SR step's sampling ({W} walkers x {S} samples x {sweeps} "
                               f"sweeps of {Ne} proposals) extrapolated from these rates"}
    return out


def projected_sampling(vmc, torch, stream, inputs, W=608, calls=2):
    """Momentum projection at N_g = Ns on the 16x16 workload (mixed form):
    all 256 translations at K = 0 (Sec. 3.2.2, Eq. momP; App. A signs), one
    M_g^-1 per translation per walker in HBM (12.8 MB per walker; 608
    walkers fill the kernel's four CTAs per SM).  Timed with CUDA events on
    the stream: vmc_sample(0, 1, 1) calls (one sweep and one measurement per
    walker, with the periodic rebuilds of every M_g^-1); then, per kernel
    launch, one sweep-only and one measurement-only call.
    Roofline of the projected sweep on its algorithmic bytes, what the fast
    updates must move with every M_g^-1 in HBM (per operation g, 4-byte
    words): a tested hop reads a row or column (N); a tested exchange forms
    R^T M_g^-1 and reads row m (N^2 + 2N); an accepted hop reads M_g^-1 for
    R^T M_g^-1 or M_g^-1 C, then reads and writes it in the update (3 N^2); an
    accepted exchange forms both products (4 N^2 with the update)."""
    prob = inputs.square16_hubbard()
    perm, sign = inputs.translation_ops(prob.lat)
    G, N = perm.shape[0], prob.N
    ctx = vmc.Context(prob, W, seed=7, precision=vmc.MIXED, max_samples=1,
                      stream=stream.cuda_stream)
    ctx.set_projection(perm, sign, np.full(G, 1.0 / G))
    ctx.sample(1, 0, 0)
    ctx.enable_timing(True)
    ctx.kernel_times()
    s0 = ctx.measure()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(calls):
        ctx.sample(0, 1, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = ctx.kernel_times()
    s1 = ctx.measure()
    ctx.sample(1, 0, 0)                     # sweep only
    kt_s = ctx.kernel_times()
    s2 = ctx.measure()
    ctx.sample(0, 1, 0)                     # measurement only
    kt_m = ctx.kernel_times()
    grid, per_sm, smem = ctx.sweep_launch()
    ctx.close()
    props = s1["n_proposals"] - s0["n_proposals"]
    acc = s1["n_accepted"] - s0["n_accepted"]
    d = {k: s2[k] - s1[k] for k in ("n_hop_tested", "n_exchange_tested", "n_hop_accepted",
                                    "n_exchange_accepted", "n_proposals")}
    sweep_ms = kt_s["sweep"][0] / max(kt_s["sweep"][1], 1)
    b = 4.0 * G * (N * d["n_hop_tested"] + (N * N + 2 * N) * d["n_exchange_tested"]
                   + 3 * N * N * d["n_hop_accepted"] + 4 * N * N * d["n_exchange_accepted"])
    hbm, src = hbm_peak_gbs()
    ach = b / (sweep_ms * 1e-3) / 1e9
    return {"walkers": W, "operations": G, "characters": "K = 0", "calls": calls,
            "ms_per_call": ms / calls, "proposals_per_s": props / (ms * 1e-3),
            "sweep_kernel_ms_per_launch": kt["sweep"][0] / max(kt["sweep"][1], 1),
            "sweep_only_ms": sweep_ms,
            "measurement_only_ms": kt_m["sweep"][0] / max(kt_m["sweep"][1], 1),
            "rebuild_ms_per_call": kt["init"][0] / calls,
            "acceptance": acc / max(props, 1), "sweep_launch": {"grid": grid, "ctas_per_sm": per_sm,
                                                                "smem_bytes": smem},
            "sweep_counts": d,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": None,
                         "kernel": "k_proj_sample<float> (sweep-only launch)",
                         "algorithmic_bytes_per_launch": b,
                         "bytes_rule": "4 N_g (N hops tested + (N^2 + 2N) exchanges tested + "
                                       "3 N^2 hops accepted + 4 N^2 exchanges accepted)",
                         "peak_source": src}}


def lanczos_moments_timing(vmc, torch, stream, inputs, W=1024, calls=3):
    """First-step power-Lanczos moments (Sec. 3.4) on the 16x16 workload,
    mixed form: vmc_lanczos_moments on the walkers' current configurations,
    CUDA events on the stream around each call.  Roofline of its table
    products (Gu, Gd: Ns N^2 FMA each; T: Ns^2 N FMA, per walker) against the
    FP32 peak; the two-move ratios (first term x second term, O(1) each from
    the tables) come on top."""
    prob = inputs.square16_hubbard()
    ctx = vmc.Context(prob, W, seed=17, precision=vmc.MIXED, max_samples=1,
                      stream=stream.cuda_stream)
    ctx.sample(4, 0, 0)
    ctx.lanczos_moments()                  # device scratch
    ms = []
    for _ in range(calls):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, h = ctx.lanczos_moments()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctx.close()
    t = statistics.median(ms)
    N, Ns = prob.N, prob.Ns
    fl = 2.0 * (2 * Ns * N * N + Ns * Ns * N) * W
    ach = fl / (t * 1e-3) / 1e12
    try:
        a, e1 = vmc.lanczos_alpha(h)
        e1 /= Ns
    except vmc.VmcError:                   # no real stationary point of E_1(alpha)
        a = e1 = None
    return {"walkers": W, "ms_per_call": t, "configurations_per_s": W / (t * 1e-3),
            "alpha_1": a, "E1_per_site": e1, "h1_per_site": h["h1"] / Ns,
            "roofline_tables": {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                                "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                                "kernel": "k_lanczos<float> (whole call)",
                                "flops_rule": "2 (2 Ns N^2 + Ns^2 N) per walker",
                                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}}


def other_workloads(vmc, torch, stream, steps=5):
    """The other configured workloads, each timed on the device (CUDA events
    on the stream) after the headline bench:
      ring8   C1: 8-site ring, FP64, 64 walkers x 200 samples x 10 sweeps and
              one FP64 Cholesky SR step per step;
      square8 C2: 8x8, FP64, 1024 walkers x 4 samples x 1 sweep, FP64 Cholesky;
      batch64 C3: 64 independent Hubbard systems (L = 4..16) x 64 walkers, mixed
              form, FP64 recompute every 64 accepted moves, 4 samples, and
              one SR step of every system (vmc_sr_step_all, mixed solve);
      j1j2    C4: 16x16 J1-J2, full f (N_p = 65,536): 1024 walkers x 8
              samples (mixed form, proposal batch depth from the tuner), then
              one dense S build of the 8192 samples by the split-BF16
              tensor-core kernel;
      projection_16x16: sampling with all 256 translations (projected_sampling);
      kondo_L8: the L = 8 Kondo chain, sampling and an SR step (mixed form);
      lanczos_16x16: power-Lanczos moments (lanczos_moments_timing)."""
    from paper_1711_11418_gb300 import inputs
    res = {}

    def timed(ctx, step, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0 = sum(ctx.measure(k)["n_proposals"] for k in range(len(ctx.problems)))
        e0.record(stream)
        for _ in range(n):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        p1 = sum(ctx.measure(k)["n_proposals"] for k in range(len(ctx.problems)))
        ms = e0.elapsed_time(e1)
        return {"ms_per_step": ms / n, "proposals_per_s": (p1 - p0) / (ms * 1e-3), "steps": n}

    sr64 = dict(dtau=0.05, shift_rel=1e-3, shift_abs=0.0, solver=vmc.CHOLESKY)
    for name, prob, W, S, sweeps in (("ring8", inputs.ring8_hubbard(), 64, 200, 10),
                                     ("square8", inputs.square8_hubbard(), 1024, 4, 1)):
        ctx = vmc.Context(prob, W, seed=11, precision=vmc.FP64, max_samples=S,
                          stream=stream.cuda_stream)
        ctx.sample(10, 0, 0)

        def step(ctx=ctx, S=S, sweeps=sweeps):
            ctx.sample(0, S, sweeps)
            ctx.sr_step(**sr64)
        step()
        res[name] = timed(ctx, step, steps) | {
            "walkers": W, "samples_per_walker": S, "sweeps_between": sweeps, "dtype": "f64",
            "energy_per_site": ctx.measure()["energy"] / prob.Ns}
        ctx.close()
    probs = inputs.batched_hubbard()
    ctx = vmc.Context(probs, 64, seed=5, precision=vmc.MIXED, max_samples=4, recompute_every=64,
                      stream=stream.cuda_stream)
    ctx.sample(10, 0, 0)

    def step_b():
        ctx.sample(0, 4, 1)
        ctx.sr_step_all(0.05, 1e-3, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-12)
    step_b()
    res["batch64"] = timed(ctx, step_b, steps) | {
        "systems": len(probs), "walkers_per_system": 64, "samples_per_walker": 4,
        "sizes_L": sorted({int(round(p.Ns ** 0.5)) for p in probs}), "dtype": "f32+f64"}
    ctx.close()
    res["projection_16x16"] = projected_sampling(vmc, torch, stream, inputs)
    # Kondo lattice, Table Kondo's L = 8 chain (16 sites, 8 of them local
    # spins): sampling and one SR step per step, mixed form
    prob = inputs.kondo_chain(8)
    ctx = vmc.Context(prob, 1024, seed=13, precision=vmc.MIXED, max_samples=8,
                      stream=stream.cuda_stream)
    ctx.sample(20, 0, 0)

    def step_k():
        ctx.sample(0, 8, 2)
        ctx.sr_step(0.05, 1e-3, 1e-4, solver=vmc.CHOLESKY)
    step_k()
    res["kondo_L8"] = timed(ctx, step_k, steps) | {
        "walkers": 1024, "samples_per_walker": 8, "sweeps_between": 2, "dtype": "f32+f64",
        "energy_per_cell": ctx.measure()["energy"] / 8}
    ctx.close()
    res["lanczos_16x16"] = lanczos_moments_timing(vmc, torch, stream, inputs)
    prob = inputs.j1j2_heisenberg()
    ctx = vmc.Context(prob, 1024, seed=3, precision=vmc.MIXED, max_samples=8,
                      stream=stream.cuda_stream)
    ctx.sample(2, 0, 0)
    # sampling: every proposal an exchange (an O(N^2) ratio), the batch depth
    # picked by the tuner; one sampling call of 8 samples timed on the stream
    b_chosen, b_ms = ctx.tune_proposal_batch(sweeps=2, candidates=(1, 2, 4, 8))
    s0 = ctx.measure()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.sample(0, 8, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    props = ctx.measure()["n_proposals"] - s0["n_proposals"]
    sampling = {"walkers": 1024, "samples_per_walker": 8, "sweeps_between": 1,
                "dtype": "f32+f64", "ms": ms_s, "proposals_per_s": props / (ms_s * 1e-3),
                "proposal_batch": b_chosen, "ms_per_sweep_by_batch": b_ms}
    ctx.enable_timing(True)
    ctx.kernel_times()
    rep = ctx.sr_step(0.05, 1e-4, 0.0, solver=vmc.CG_DENSE, cg_eps=1e-3, cg_kmax=1)
    ms = ctx.kernel_times()["sr_gemm"][0]
    rows, Np = 1024 * 8, prob.Np
    fl = float(rows) * Np * Np                       # N_MC N_p^2 (symmetric product)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    pk = peaks.get("bf16_tflops", 1900.0)
    res["j1j2"] = {"rows": rows, "Np": Np, "s_build_ms": ms,
                   "s_kernel": vmc.S_KERNELS[rep["s_kernel"]],
                   "tflops_method": fl / (ms * 1e-3) / 1e12,
                   "tflops_three_products": 3 * fl / (ms * 1e-3) / 1e12,
                   "frac_method": fl / (ms * 1e-3) / 1e12 / pk,
                   "frac_three_products": 3 * fl / (ms * 1e-3) / 1e12 / pk,
                   "peak_tflops": pk, "peak_source": "measured bf16 burst" if peaks else "fallback",
                   "flops_rule": "method: N_MC N_p^2 (the symmetric product once); three "
                                 "products: split-BF16 hi.hi + hi.lo + lo.hi",
                   "sampling": sampling}
    ctx.close()
    return res


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


def sweep_bytes(d, N, esize):
    """Algorithmic bytes of the update sweep (A3-A6) from its counters: the
    block M^-1 read and written once per accepted move (2 esize N^2) and one
    block column plus one gathered f row per proposal (2 esize N)."""
    return 2.0 * esize * N * N * d["n_accepted"] + 2.0 * esize * N * d["n_proposals"]


def energy_statistics(vmc, prob, params, ele0, walkers, samples, recompute, stream):
    """Statistical half of "equal energy accuracy": the plain FP64 and the
    mixed form sample the same wave function (fixed parameters, no SR in
    between) from the same configurations with the same proposal streams,
    `samples` measurements each after one sweep.  Each form's energy per site
    carries a standard error from its per-walker means (walkers are
    independent chains).  Walkers whose two chains end in the same
    configuration made the same decisions throughout, so their rows compare
    the two precisions on identical configurations at every sample, i.e. at
    several points between the mixed form's FP64 rebuilds."""
    Ns = prob.Ns
    E, ele = {}, {}
    for name, prec in (("fp64", vmc.FP64), ("mixed", vmc.MIXED)):
        ctx = vmc.Context(prob.copy_with(params=params), walkers, seed=777, precision=prec,
                          max_samples=samples,
                          recompute_every=recompute if prec == vmc.MIXED else -1, stream=stream)
        ctx.set_configs(ele0)
        ctx.sample(0, samples, 1)
        E[name] = ctx.get_samples(with_O=False)[0].reshape(walkers, samples) / Ns
        ele[name] = ctx.get_configs()[0]
        ctx.close()
    wm = {k: v.mean(axis=1) for k, v in E.items()}
    e = {k: float(v.mean()) for k, v in wm.items()}
    se = {k: float(v.std(ddof=1) / math.sqrt(walkers)) for k, v in wm.items()}
    sig = math.sqrt(se["fp64"] ** 2 + se["mixed"] ** 2)
    diff = e["mixed"] - e["fp64"]
    paired = wm["mixed"] - wm["fp64"]
    same = (ele["fp64"] == ele["mixed"]).all(axis=1)
    d = abs(E["mixed"] - E["fp64"])[same]
    return {"fp64_energy_per_site": e["fp64"], "mixed_energy_per_site": e["mixed"],
            "stderr_fp64": se["fp64"], "stderr_mixed": se["mixed"], "sigma_combined": sig,
            "difference": diff, "within_3sigma": abs(diff) <= 3 * sig,
            "within_1e-4": abs(diff) <= 1e-4,
            "paired_stderr": float(paired.std(ddof=1) / math.sqrt(walkers)),
            "walkers": walkers, "samples_per_walker": samples, "sweeps_between": 1,
            "mixed_recompute_every_accepted": recompute,
            "walkers_same_chain": int(same.sum()),
            "same_chain_dE_per_site_max_by_sample": [float(x) for x in d.max(axis=0)] if d.size else None,
            "same_chain_dE_per_site_p99": float(np.percentile(d, 99)) if d.size else None,
            "same_chain_entries_over_1e-4": int((d > 1e-4).sum()),
            "how": "both forms, same parameters, same starting configurations and proposal "
                   "streams, no SR in between; standard errors from per-walker means"}


def delta(a, b):
    return {k: b[k] - a[k] for k in b if isinstance(b[k], int)}


def run_arm(vmc, prob, args, precision, stream, torch, world, rebuild=0):
    W, S = args.walkers, args.samples
    ctx = vmc.Context(prob, W, seed=1234 + int(os.environ.get("RANK", 0)), precision=precision,
                      max_samples=S, recompute_every=args.recompute if precision == vmc.MIXED else -1,
                      stream=stream.cuda_stream, rebuild=rebuild)
    ctx.sample(args.equil, 0, 0)                        # equilibration (untimed)
    # proposal batch depth picked by the library's tuner (sweeps only, untimed)
    b_chosen, b_ms = ctx.tune_proposal_batch(sweeps=2, candidates=(1, 2, 4, 8))
    pbatch = {"chosen": b_chosen, "ms_per_sweep": b_ms}
    # Immediate updates: they keep the mixed form's double-float inverse (the
    # delayed form keeps FP32 words only, so it is not used at the accuracy
    # this bench checks).
    delay = {"chosen": 1, "why": "immediate updates keep the double-float inverse"}
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
    grid, per_sm, smem = ctx.sweep_launch()
    return ctx, dict(ms=ms, stats=d, kt=kt, launches=launches, clocks=clk,
                     energy=statistics.fmean(energies), last=st1, solve=solve,
                     props_all=props_all, sr=sr, delay=delay, pbatch=pbatch,
                     launch={"grid": grid, "ctas_per_sm": per_sm, "smem_bytes": smem})


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
        # the mixed form with its opt-in double-float rebuild, same step
        dfr = None
        if not args.no_df_rebuild:
            ctxdf, dfr = run_arm(vmc, prob, args, vmc.MIXED, stream, torch, world,
                                 rebuild=vmc.REBUILD_DOUBLE_FLOAT)
            ctxdf.close()
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
        stat = None
        if not args.no_fp64:
            stat = energy_statistics(vmc, prob, params, ele, args.walkers, args.stat_samples,
                                     args.recompute, stream.cuda_stream)
        # The update sweep alone (A3-A6: proposals, ratios, accepted updates;
        # no measurement): sweep-only launches of the mixed context, timed by
        # the library's CUDA events on the stream, after the timed region.
        ctx.kernel_times()
        sw0 = ctx.measure()
        for _ in range(args.sweep_only):
            ctx.sample(1, 0, 0)
        kt_sw = ctx.kernel_times()
        sw = delta(sw0, ctx.measure())
        # End to end: parameters from pinned host memory, energy and parameters back
        e2e = None
        if not args.no_e2e:
            hp = torch.empty(prob.Np, dtype=torch.float64, pin_memory=True).numpy()
            hp[:] = params
            t0 = time.perf_counter()
            m0 = ctx.measure()
            p0 = m0["n_proposals"]
            for _ in range(args.steps):
                ctx.set_params(hp)
                ctx.sample(0, args.samples, 1)
                ctx.sr_step(**mixed["sr"])
                hp[:] = ctx.get_params()
                _ = ctx.measure()["energy"]
            torch.cuda.synchronize()
            dt = reduce_over_ranks(torch, time.perf_counter() - t0, "max")
            m1 = ctx.measure()
            props = reduce_over_ranks(torch, m1["n_proposals"] - p0, "sum")
            # run after the timed region, further along the SR trajectory:
            # its acceptance (accepted moves are the costly part) beside it
            e2e = {"value": props / dt, "unit": "proposals/s",
                   "h2d_bytes_per_step": 8 * prob.Np,
                   "d2h_bytes_per_step": 8 * prob.Np + 8 * args.walkers * args.samples + 64,
                   "ms_per_step": 1e3 * dt / args.steps,
                   "acceptance": (m1["n_accepted"] - m0["n_accepted"]) / max(m1["n_proposals"] - p0, 1)}
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
        others = None if args.no_others else other_workloads(vmc, torch, stream)

    def summarize(r):
        d = r["stats"]
        secs = r["ms"] * 1e-3
        sweep_ms, sweep_n = r["kt"]["sweep"]
        return {"proposals_per_s": r["props_all"] / secs, "ms_per_step": r["ms"] / args.steps,
                "sweep_kernel_ms_per_launch": sweep_ms / max(sweep_n, 1), "sweep_launches": sweep_n,
                "init_ms_per_step": r["kt"]["init"][0] / args.steps,
                "sr_ms_per_step": r["kt"]["sr"][0] / args.steps,
                "acceptance": d["n_accepted"] / max(d["n_proposals"], 1),
                "accepted_per_s": r["props_all"] / secs * d["n_accepted"] / max(d["n_proposals"], 1),
                "energy_per_site": r["energy"] / prob.Ns, "recomputes": d["n_recomputes"],
                "sr_solve": r["solve"], "delay_tuner": r["delay"], "proposal_batch_tuner": r["pbatch"],
                "sweep_launch": r["launch"]}

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
    # Survey roofline of the update sweep: algorithmic bytes (the FP32 block
    # streamed per accepted move, a column and an f row per proposal) per
    # launch / launch time, against the measured HBM copy bandwidth.  The
    # launch also measures E_loc and O_k (not counted in these bytes).
    b_launch = sweep_bytes(mixed["stats"], N, 4) / max(sweep_n, 1)
    ach_b = b_launch / t_launch / 1e9
    ach = f32 / max(sweep_n, 1) / t_launch / 1e12
    roof_sweep = {"bound": "hbm", "achieved": ach_b, "peak": hbm, "unit": "GB/s",
                  "frac": ach_b / hbm, "traffic": None,
                  "kernel": "k_sample<float> (sweep + measurement)",
                  "algorithmic_bytes_per_launch": b_launch,
                  "bytes_rule": "2 x 4 x N^2 per accepted move + 2 x 4 x N per proposal (N = 112)",
                  "ms_in_timed_region": sweep_ms, "ms_per_launch": t_launch * 1e3,
                  "peak_source": hbm_src,
                  "alu": {"achieved_tflops": ach, "peak_tflops": FP32_PEAK_TFLOPS,
                          "frac": ach / FP32_PEAK_TFLOPS,
                          "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}}
    sw_ms, sw_n = kt_sw["sweep"]
    t_sw = sw_ms * 1e-3 / max(sw_n, 1)
    b_sw = sweep_bytes(sw, N, 4) / max(sw_n, 1)
    roof_sweep_only = {"bound": "hbm", "achieved": b_sw / t_sw / 1e9, "peak": hbm, "unit": "GB/s",
                       "frac": b_sw / t_sw / 1e9 / hbm, "kernel": "k_sample<float>, sweeps only",
                       "traffic": TRAFFIC_SWEEP_ONLY_4096 * scale,
                       "launches": sw_n, "ms_per_launch": t_sw * 1e3,
                       "algorithmic_bytes_per_launch": b_sw,
                       "acceptance": sw["n_accepted"] / max(sw["n_proposals"], 1),
                       "proposals_per_s": sw["n_proposals"] / max(sw_ms * 1e-3, 1e-12),
                       "what": "the update sweep alone (A3-A6), one sweep per launch, "
                               "timed after the timed region on the same context"}
    init_ms, _ = mixed["kt"]["init"]
    n_inv = args.steps * args.walkers + mixed["stats"]["n_recomputes"]
    ach_init = 2.0 * N ** 3 * n_inv / max(init_ms * 1e-3, 1e-12) / 1e12
    roof_init = {"bound": "alu", "achieved": ach_init, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                 "frac": ach_init / FP64_PEAK_TFLOPS, "traffic": TRAFFIC_INIT_4096 * scale,
                 "traffic_launch": "the full rebuild of all walkers after an SR step",
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
        "mixed_double_float_rebuild": dict(
            summarize(dfr), what="the same step with the mixed form's opt-in double-float "
            "from-scratch inverses (VMC_REBUILD_DOUBLE_FLOAT) instead of FP64 ones") if dfr else None,
        "energy_check": {"same_configs_dE_per_site_mean": dE, "same_configs_dE_per_site_max": dE_max,
                         "same_configs_dE_per_site_p99": dE_p99,
                         "walkers_over_tolerance": n_over, "walkers": args.walkers,
                         "tolerance": 1e-4,
                         "tolerance_applies_to": "the energy estimate (walker mean)",
                         "statistical": stat},
        "roofline": roof,
        "roofline_second": roof2,
        "roofline_sweep_only": roof_sweep_only,
        "pair_correlations": pair_corr,
        "other_workloads": others,
        "clocks": mixed["clocks"],
        "gpu_launches": mixed["launches"],
        "e2e": e2e,
    }
    if pool is not None:
        line["cpu_baseline"] = cpu_baseline(pool, cores, args.cpu_seconds)
        line["cpu_baseline_other"] = cpu_baseline_configs(pool, cores)
        pool.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_learned(args):
    """The learned part at its configured size: 16x16 Hubbard, U/t = 8,
    Ne = 224, the Gutzwiller-Jastrow-Pfaffian state times an MLP correlation
    factor (512 occupations -> 1024 tanh units -> 1, BF16 weights in the
    sweep, N(0, 0.01^2) initial weights), 4096 walkers, SR by SR-CG (S never
    formed, FP32 sample matrix, FP64 CG).  Two protocols with the same
    walkers, samples per step, SR steps and solver for both states:
      cold: both trained from the same initial state for `learned_steps`;
      warm: the plain state trained for `learned_steps`, then continued for
        `learned_finetune` more steps, beside the MLP state that starts from
        the trained plain parameters (and its walkers) and trains all
        527,406 parameters for the same `learned_finetune` steps.
    Afterwards each state is sampled with fixed parameters; energies per site
    with standard errors from per-walker means."""
    import torch
    from paper_1711_11418_gb300 import build, inputs, vmc
    build.build()
    torch.cuda.set_device(0)
    W, S = args.walkers, args.samples
    sr = dict(dtau=0.05, shift_rel=1e-3, shift_abs=1e-4, solver=vmc.CG, cg_eps=1e-4,
              cg_kmax=200)
    plain_p, mlp_p = inputs.square16_hubbard(), inputs.square16_hubbard_mlp(hidden=1024)

    def train(ctx, prob, steps):
        traj, iters = [], []
        for _ in range(steps):
            ctx.sample(0, S, 1)
            rep = ctx.sr_step(**sr)
            traj.append(rep["energy"] / prob.Ns)
            iters.append(rep["cg_iters"])
        return traj, iters

    def evaluate(ctx, prob):
        wm = []
        for _ in range(args.learned_eval):
            ctx.sample(0, S, 1)
            wm.append(ctx.get_samples(with_O=False)[0].reshape(W, S).mean(axis=1))
        wm = np.mean(wm, axis=0) / prob.Ns
        return float(wm.mean()), float(wm.std(ddof=1) / math.sqrt(W))

    def record(prob, e, se, t, traj, iters):
        return {"energy_per_site": e, "stderr": se, "Np": prob.Np, "train_seconds": round(t, 2),
                "cg_iterations_mean": float(np.mean(iters)) if iters else 0.0,
                "trajectory_every_10_steps": [round(x, 6) for x in traj[::10]]}

    def gain(a, b):
        g = a["energy_per_site"] - b["energy_per_site"]
        sg = math.hypot(a["stderr"], b["stderr"])
        return {"gain_per_site": g, "gain_sigma": sg, "gain_significant_3sigma": bool(g > 3 * sg)}

    out = {}
    # cold start: both from the same initial state
    cold = {}
    plain_ctx = None
    for name, prob in (("plain", plain_p), ("mlp", mlp_p)):
        t0 = time.perf_counter()
        ctx = vmc.Context(prob, W, seed=2024, precision=vmc.MIXED, max_samples=S,
                          recompute_every=args.recompute)
        ctx.sample(args.equil, 0, 0)
        traj, iters = train(ctx, prob, args.learned_steps)
        t = time.perf_counter() - t0
        e, se = evaluate(ctx, prob)
        cold[name] = record(prob, e, se, t, traj, iters)
        if name == "plain":
            plain_ctx = ctx
        else:
            ctx.close()
    out["cold"] = {**cold, **gain(cold["plain"], cold["mlp"])}
    # warm start: the MLP state from the trained plain state
    warm = {}
    if args.learned_finetune > 0:
        params = plain_ctx.get_params()
        ele, _ = plain_ctx.get_configs()
        t0 = time.perf_counter()
        traj, iters = train(plain_ctx, plain_p, args.learned_finetune)
        e, se = evaluate(plain_ctx, plain_p)
        warm["plain"] = record(plain_p, e, se, time.perf_counter() - t0, traj, iters)
        pm = mlp_p.params.copy()
        pm[:plain_p.Np] = params          # g, v, f first; the MLP block keeps its start
        t0 = time.perf_counter()
        ctx = vmc.Context(mlp_p.copy_with(params=pm), W, seed=2025, precision=vmc.MIXED,
                          max_samples=S, recompute_every=args.recompute)
        ctx.set_configs(ele)
        traj, iters = train(ctx, mlp_p, args.learned_finetune)
        e, se = evaluate(ctx, mlp_p)
        warm["mlp"] = record(mlp_p, e, se, time.perf_counter() - t0, traj, iters)
        ctx.close()
        out["warm"] = {**warm, **gain(warm["plain"], warm["mlp"])}
    plain_ctx.close()
    print(json.dumps({"what": "learned part: plain Gutzwiller-Jastrow-Pfaffian vs x MLP "
                              "correlation factor, same sample budget",
                      "workload": "hubbard_16x16_U8_Ne224_apbc, MLP 512->1024->1",
                      "walkers": W, "samples_per_step": W * S,
                      "sr_steps": args.learned_steps, "finetune_steps": args.learned_finetune,
                      "sr": {k: v for k, v in sr.items() if k != "solver"} | {"solver": "sr_cg"},
                      "eval_samples_per_walker": args.learned_eval * S, **out}))


def main():
    args = parse()
    if args.learned:
        run_learned(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
