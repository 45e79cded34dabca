"""The two calculation modes of the flow of Sec. 2.2.3 as loops over a
``vmc.Context``, with one JSON record per step.

* ``optimize``: NVMCCalMode = 0 -- sample, then one SR step (Sec. 3.3), per
  step; the record holds the energy estimate, its error from the
  per-walker means, the acceptance, the inverse drift and the solver's
  report.
* ``measure_physics``: NVMCCalMode = 1 -- with fixed parameters, advance
  the chains and measure the pair correlations (``Context.measure_corr``)
  a number of times; returns their mean over the measurements and the
  standard error of that mean.

Orchestration only: every sampled quantity, ratio and solve comes from the
library's kernels through the binding; the host only averages the
library's per-measurement results.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

RECORD_STATS = ("energy", "variance", "stderr_walkers", "acceptance", "max_drift",
                "n_flagged", "n_recomputes")
RECORD_SR = ("norm_g", "norm_dalpha", "cg_iters", "rel_residual", "fallback")


def _writer(log):
    if log is None:
        return None, lambda rec: None
    f = open(log, "a") if isinstance(log, str) else log

    def write(rec):
        f.write(json.dumps(rec) + "\n")
        f.flush()
    return (f if isinstance(log, str) else None), write


def optimize(ctx, n_steps, n_samples, sweeps_between=1, n_warmup=10, dtau=0.05,
             shift_rel=1e-3, shift_abs=0.0, solver=0, cg_eps=1e-10, cg_kmax=1000,
             system=0, log=None):
    """n_steps times: ``ctx.sample`` (n_warmup sweeps before the first
    step only), ``ctx.measure``, ``ctx.sr_step``.  Returns the records;
    with ``log`` (a path or a text file object) each is also appended as
    one JSON line."""
    own, write = _writer(log)
    records = []
    try:
        for step in range(n_steps):
            t0 = time.perf_counter()
            ctx.sample(n_warmup if step == 0 else 0, n_samples, sweeps_between)
            st = ctx.measure(system)
            rep = ctx.sr_step(dtau, shift_rel, shift_abs, solver=solver, cg_eps=cg_eps,
                              cg_kmax=cg_kmax, system=system)
            rec = {"mode": "optimize", "step": step, "system": system}
            rec.update({k: st[k] for k in RECORD_STATS if k in st})
            rec.update({"sr_" + k: rep[k] for k in RECORD_SR if k in rep})
            rec["seconds"] = time.perf_counter() - t0
            records.append(rec)
            write(rec)
    finally:
        if own is not None:
            own.close()
    return records


def measure_physics(ctx, n_measurements, sweeps_between=1, n_warmup=0, system=0, log=None):
    """n_measurements times: advance every chain by ``sweeps_between``
    sweeps (``ctx.sample(sweeps_between, 0, 0)``: sweeps only, so no E_loc
    or O_k row is measured and the stored samples of an earlier ``optimize``
    step are left as they were), then ``ctx.measure_corr``.  Returns
    (mean [6, Ns, Ns], standard error of the mean [6, Ns, Ns], records).
    The error treats the measurements as independent; with
    sweeps_between >= the autocorrelation time it is the Monte Carlo
    error of Eq. MC's estimate."""
    if n_measurements < 1:
        raise ValueError("n_measurements must be >= 1")
    own, write = _writer(log)
    records = []
    acc = acc2 = None
    try:
        if n_warmup:
            ctx.sample(n_warmup, 0, 0)
        for k in range(n_measurements):
            t0 = time.perf_counter()
            ctx.sample(sweeps_between, 0, 0)
            c = np.asarray(ctx.measure_corr(system=system), np.float64)
            acc = c.copy() if acc is None else acc + c
            acc2 = c * c if acc2 is None else acc2 + c * c
            rec = {"mode": "measure", "measurement": k, "system": system,
                   "doublons_per_site": float(0.5 * (np.trace(c[2]) - np.trace(c[0])
                                                     - np.trace(c[1])) / c.shape[-1]),
                   "seconds": time.perf_counter() - t0}
            records.append(rec)
            write(rec)
    finally:
        if own is not None:
            own.close()
    n = n_measurements
    mean = acc / n
    if n > 1:
        var = np.maximum(acc2 / n - mean * mean, 0.0) * n / (n - 1)
        err = np.sqrt(var / n)
    else:
        err = np.full_like(mean, math.nan)
    return mean, err, records
