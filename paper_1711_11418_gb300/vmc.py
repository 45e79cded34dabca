"""ctypes binding of libvmc.so (include/vmc.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  Importing this
module does not load the library; the first Context does, and raises
``VmcError`` if ``libvmc.so`` is missing (build it with
``paper_1711_11418_gb300.build.build()``) or no CUDA device is present.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvmc.so")

FP64, MIXED = 0, 1
REBUILD_FP64, REBUILD_DOUBLE_FLOAT = 0, 1
FORCE_STATIC_MAX_DOUBLES = 1 << 20
CHOLESKY, CG, CG_DENSE, MIXED_IR = 0, 1, 2, 3
S_KERNELS = ("none", "fp64_simt", "tcgen05_tma_persistent", "tcgen05_tiles")
CORR_KINDS = ("cdag_c_up", "cdag_c_dn", "n_n", "sz_sz", "sp_sm", "s_s")
_I32P = C.POINTER(C.c_int32)
_F64P = C.POINTER(C.c_double)
_I8P = C.POINTER(C.c_int8)
_U64P = C.POINTER(C.c_uint64)


class VmcModel(C.Structure):
    _fields_ = [("Ns", C.c_int32), ("n_hop", C.c_int32), ("hop_i", _I32P), ("hop_j", _I32P),
                ("hop_t", _F64P), ("U", _F64P), ("n_V", C.c_int32), ("V_i", _I32P),
                ("V_j", _I32P), ("V_val", _F64P), ("n_J", C.c_int32), ("J_i", _I32P),
                ("J_j", _I32P), ("J_val", _F64P), ("local_spin", C.c_int32),
                ("local_site", _I8P)]


class VmcLayout(C.Structure):
    _fields_ = [("n_g", C.c_int32), ("n_v", C.c_int32), ("n_f", C.c_int32),
                ("g_idx", _I32P), ("v_idx", _I32P), ("f_idx", _I32P), ("f_sign", _I8P),
                ("n_hidden", C.c_int32)]


class VmcOpts(C.Structure):
    _fields_ = [("n_walkers", C.c_int32), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("delay_k", C.c_int32), ("recompute_every", C.c_int32),
                ("max_samples", C.c_int32), ("stream", C.c_void_p), ("rebuild", C.c_int32)]


class VmcStats(C.Structure):
    _fields_ = [("energy", C.c_double), ("variance", C.c_double),
                ("stderr_walkers", C.c_double), ("acceptance", C.c_double),
                ("n_proposals", C.c_int64), ("n_accepted", C.c_int64),
                ("n_samples", C.c_int32), ("n_flagged", C.c_int32), ("max_drift", C.c_double),
                ("n_hop_tested", C.c_int64), ("n_exchange_tested", C.c_int64),
                ("n_hop_accepted", C.c_int64), ("n_exchange_accepted", C.c_int64),
                ("n_recomputes", C.c_int64), ("n_measured_hops", C.c_int64),
                ("n_measured_exchanges", C.c_int64), ("n_measurements", C.c_int64)]


class VmcSrOpts(C.Structure):
    _fields_ = [("dtau", C.c_double), ("shift_rel", C.c_double), ("shift_abs", C.c_double),
                ("solver", C.c_int32), ("cg_eps", C.c_double), ("cg_kmax", C.c_int32)]


class VmcSrReport(C.Structure):
    _fields_ = [("energy", C.c_double), ("norm_g", C.c_double), ("norm_dalpha", C.c_double),
                ("cg_iters", C.c_int32), ("n_params", C.c_int32), ("rel_residual", C.c_double),
                ("fallback", C.c_int32), ("s_kernel", C.c_int32)]


class VmcError(RuntimeError):
    def __init__(self, code, where=""):
        msg = _lib.vmc_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


_lib = None
EXPORTS = ["vmc_create", "vmc_create_batch", "vmc_destroy", "vmc_strerror", "vmc_set_configs",
           "vmc_get_configs", "vmc_sample", "vmc_measure", "vmc_get_samples", "vmc_set_samples",
           "vmc_sr_step", "vmc_get_sr_matrices", "vmc_get_params", "vmc_set_params",
           "vmc_num_params", "vmc_eval_ratios", "vmc_get_inverse", "vmc_kernel_launches",
           "vmc_enable_timing", "vmc_kernel_times", "vmc_sr_force_static", "vmc_set_delay",
           "vmc_get_delay", "vmc_tune_delay", "vmc_sr_step_all", "vmc_measure_corr",
           "vmc_test_stall", "vmc_set_projection", "vmc_lanczos_moments", "vmc_lanczos_alpha",
           "vmc_sweep_launch", "vmc_set_proposal_batch", "vmc_get_proposal_batch",
           "vmc_tune_proposal_batch"]
STALL_NONE, STALL_SAMPLE, STALL_S_BUILD = 0, 1, 2


def load(path: str = LIB_PATH):
    """Load libvmc.so and declare the signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise VmcError(-3, f"libvmc.so not found at {path}; build it first")
    L = C.CDLL(path)
    P = C.c_void_p
    L.vmc_create.argtypes = [C.POINTER(P), C.POINTER(VmcModel), C.c_int32, C.POINTER(VmcLayout),
                             _F64P, C.c_double, C.POINTER(VmcOpts)]
    L.vmc_create_batch.argtypes = [C.POINTER(P), C.c_int32, C.POINTER(VmcModel), _I32P,
                                   C.POINTER(VmcLayout), C.POINTER(_F64P), _F64P,
                                   C.POINTER(VmcOpts)]
    L.vmc_destroy.argtypes = [P]
    L.vmc_destroy.restype = None
    L.vmc_strerror.argtypes = [C.c_int]
    L.vmc_strerror.restype = C.c_char_p
    L.vmc_set_configs.argtypes = [P, C.c_int32, _I32P, _U64P]
    L.vmc_get_configs.argtypes = [P, C.c_int32, _I32P, _U64P]
    L.vmc_sample.argtypes = [P, C.c_int32, C.c_int32, C.c_int32]
    L.vmc_measure.argtypes = [P, C.c_int32, C.POINTER(VmcStats)]
    L.vmc_measure_corr.argtypes = [P, C.c_int32, _F64P, _F64P]
    L.vmc_get_samples.argtypes = [P, C.c_int32, _F64P, _F64P]
    L.vmc_set_samples.argtypes = [P, C.c_int32, C.c_int32, _F64P, _F64P]
    L.vmc_sr_step.argtypes = [P, C.c_int32, C.POINTER(VmcSrOpts), C.POINTER(VmcSrReport)]
    L.vmc_sr_step_all.argtypes = [P, C.POINTER(VmcSrOpts), C.POINTER(VmcSrReport)]
    L.vmc_get_sr_matrices.argtypes = [P, C.c_int32, C.c_double, C.c_double, _F64P, _F64P]
    L.vmc_get_params.argtypes = [P, C.c_int32, _F64P]
    L.vmc_set_params.argtypes = [P, C.c_int32, _F64P]
    L.vmc_num_params.argtypes = [P, C.c_int32]
    L.vmc_eval_ratios.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, _I32P, _F64P]
    L.vmc_get_inverse.argtypes = [P, C.c_int32, C.c_int32, _F64P, _F64P, _I32P]
    L.vmc_enable_timing.argtypes = [P, C.c_int32]
    L.vmc_kernel_times.argtypes = [P, _F64P, C.POINTER(C.c_int64)]
    L.vmc_sr_force_static.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P]
    L.vmc_kernel_launches.argtypes = [P]
    L.vmc_kernel_launches.restype = C.c_int64
    L.vmc_set_delay.argtypes = [P, C.c_int32]
    L.vmc_get_delay.argtypes = [P]
    L.vmc_tune_delay.argtypes = [P, C.c_int32, _I32P, C.c_int32, _I32P, _F64P]
    L.vmc_set_proposal_batch.argtypes = [P, C.c_int32]
    L.vmc_get_proposal_batch.argtypes = [P]
    L.vmc_tune_proposal_batch.argtypes = [P, C.c_int32, _I32P, C.c_int32, _I32P, _F64P]
    L.vmc_test_stall.argtypes = [P, C.c_int32, C.c_int32, C.c_int32]
    L.vmc_set_projection.argtypes = [P, C.c_int32, _I32P, _I8P, _F64P]
    L.vmc_lanczos_moments.argtypes = [P, C.c_int32, _F64P, _F64P, _F64P]
    L.vmc_lanczos_alpha.argtypes = [_F64P, _F64P, _F64P]
    L.vmc_sweep_launch.argtypes = [P, _I32P, _I32P, C.POINTER(C.c_int64)]
    for name in EXPORTS:
        if name not in ("vmc_destroy", "vmc_strerror", "vmc_kernel_launches"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None and a.size else None


def _check(code, where):
    if code != 0:
        raise VmcError(code, where)


class _Arrays:
    """Keeps the numpy arrays behind one system's structs alive."""

    def __init__(self, prob):
        i32 = lambda x: np.ascontiguousarray(x, np.int32)
        f64 = lambda x: np.ascontiguousarray(x, np.float64)
        self.hop_i, self.hop_j, self.hop_t = i32(prob.hop_i), i32(prob.hop_j), f64(prob.hop_t)
        self.U = f64(prob.U)
        self.V_i, self.V_j, self.V_val = i32(prob.V_i), i32(prob.V_j), f64(prob.V_val)
        self.J_i, self.J_j, self.J_val = i32(prob.ex_i), i32(prob.ex_j), f64(prob.ex_J)
        self.g_idx, self.v_idx = i32(prob.g_idx), i32(prob.v_idx)
        self.f_idx = i32(prob.f_idx)
        self.f_sign = np.ascontiguousarray(prob.f_sign, np.int8)
        self.params = f64(prob.params)
        ls = getattr(prob, "local_sites", None)
        self.local_site = None if ls is None else np.ascontiguousarray(np.asarray(ls, bool), np.int8)
        self.model = VmcModel(
            prob.lat.Ns, self.hop_i.size, _p(self.hop_i, _I32P), _p(self.hop_j, _I32P),
            _p(self.hop_t, _F64P), _p(self.U, _F64P), self.V_i.size, _p(self.V_i, _I32P),
            _p(self.V_j, _I32P), _p(self.V_val, _F64P), self.J_i.size, _p(self.J_i, _I32P),
            _p(self.J_j, _I32P), _p(self.J_val, _F64P), int(prob.local_spin),
            _p(self.local_site, _I8P))
        self.layout = VmcLayout(prob.n_g, prob.n_v, prob.n_f, _p(self.g_idx, _I32P),
                                _p(self.v_idx, _I32P), _p(self.f_idx, _I32P),
                                _p(self.f_sign, _I8P), int(getattr(prob, "n_hidden", 0) or 0))


class Context:
    """One vmc_ctx: a single system or a batch of systems."""

    def __init__(self, problems, n_walkers, seed=1, precision=FP64, max_samples=1,
                 delay_k=0, recompute_every=0, stream=None, rebuild=REBUILD_FP64):
        L = load()
        probs = problems if isinstance(problems, (list, tuple)) else [problems]
        self.problems = list(probs)
        self.n_walkers = int(n_walkers)
        self.precision = precision
        arrs = [_Arrays(p) for p in probs]
        opts = VmcOpts(int(n_walkers), int(seed) & 0xFFFFFFFFFFFFFFFF, int(precision),
                       int(delay_k), int(recompute_every), int(max_samples),
                       C.c_void_p(stream) if stream else None, int(rebuild))
        h = C.c_void_p()
        if len(probs) == 1:
            rc = L.vmc_create(C.byref(h), C.byref(arrs[0].model), int(probs[0].Ne),
                              C.byref(arrs[0].layout), _p(arrs[0].params, _F64P),
                              float(probs[0].p_exchange), C.byref(opts))
        else:
            n = len(probs)
            models = (VmcModel * n)(*[a.model for a in arrs])
            layouts = (VmcLayout * n)(*[a.layout for a in arrs])
            ne = np.array([p.Ne for p in probs], np.int32)
            pp = (_F64P * n)(*[_p(a.params, _F64P) for a in arrs])
            pex = np.array([p.p_exchange for p in probs], np.float64)
            rc = L.vmc_create_batch(C.byref(h), n, models, _p(ne, _I32P), layouts, pp,
                                    _p(pex, _F64P), C.byref(opts))
        _check(rc, "vmc_create")
        self._h = h
        self._L = L

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._L.vmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configurations
    def set_configs(self, ele, system=0, counters=None):
        p = self.problems[system]
        ele = np.ascontiguousarray(ele, np.int32).reshape(self.n_walkers, p.Ne)
        ctr = None if counters is None else np.ascontiguousarray(counters, np.uint64)
        _check(self._L.vmc_set_configs(self._h, system, _p(ele, _I32P),
                                       _p(ctr, _U64P) if ctr is not None else None),
               "vmc_set_configs")

    def get_configs(self, system=0):
        p = self.problems[system]
        ele = np.zeros((self.n_walkers, p.Ne), np.int32)
        ctr = np.zeros(self.n_walkers, np.uint64)
        _check(self._L.vmc_get_configs(self._h, system, _p(ele, _I32P), _p(ctr, _U64P)),
               "vmc_get_configs")
        return ele, ctr

    # -- sampling and measurement
    def sample(self, n_warmup, n_samples, sweeps_between):
        _check(self._L.vmc_sample(self._h, int(n_warmup), int(n_samples), int(sweeps_between)),
               "vmc_sample")

    def measure(self, system=0):
        s = VmcStats()
        _check(self._L.vmc_measure(self._h, system, C.byref(s)), "vmc_measure")
        return {k: getattr(s, k) for k, _ in VmcStats._fields_}

    def measure_corr(self, system=0, timing=False):
        """Pair correlations of the walkers' current configurations
        (vmc_measure_corr): array [6, Ns, Ns] indexed [kind, i, j] (kinds
        CORR_KINDS).  With timing=True also returns (ratio-kernel ms,
        whole-measurement ms)."""
        Ns = self.problems[system].Ns
        out = np.zeros((6, Ns, Ns))
        ms = np.zeros(2)
        _check(self._L.vmc_measure_corr(self._h, system, _p(out, _F64P),
                                        _p(ms, _F64P) if timing else None), "vmc_measure_corr")
        return (out, (float(ms[0]), float(ms[1]))) if timing else out

    def num_params(self, system=0):
        n = self._L.vmc_num_params(self._h, system)
        if n < 0:
            raise VmcError(n, "vmc_num_params")
        return n

    def get_samples(self, system=0, rows=None, with_O=True):
        """Stored samples (vmc_get_samples): E [rows] and O [rows, Np] (None
        when with_O is False: only E is copied)."""
        st = self.measure(system)
        rows = st["n_samples"] if rows is None else rows
        Np = self.num_params(system)
        E = np.zeros(rows)
        O = np.zeros((rows, Np)) if with_O else None
        _check(self._L.vmc_get_samples(self._h, system, _p(E, _F64P),
                                       _p(O, _F64P) if with_O else None), "vmc_get_samples")
        return E, O

    def set_samples(self, E, O, system=0):
        E = np.ascontiguousarray(E, np.float64)
        O = np.ascontiguousarray(O, np.float64)
        _check(self._L.vmc_set_samples(self._h, system, E.size, _p(E, _F64P), _p(O, _F64P)),
               "vmc_set_samples")

    # -- SR
    def sr_step(self, dtau, shift_rel=0.0, shift_abs=0.0, solver=CHOLESKY, cg_eps=1e-10,
                cg_kmax=1000, system=0):
        o = VmcSrOpts(dtau, shift_rel, shift_abs, solver, cg_eps, cg_kmax)
        r = VmcSrReport()
        _check(self._L.vmc_sr_step(self._h, system, C.byref(o), C.byref(r)), "vmc_sr_step")
        return {k: getattr(r, k) for k, _ in VmcSrReport._fields_}

    def sr_step_all(self, dtau, shift_rel=0.0, shift_abs=0.0, solver=CHOLESKY, cg_eps=1e-10,
                    cg_kmax=1000):
        """One SR step for every system (vmc_sr_step_all); a report per system."""
        o = VmcSrOpts(dtau, shift_rel, shift_abs, solver, cg_eps, cg_kmax)
        reps = (VmcSrReport * len(self.problems))()
        _check(self._L.vmc_sr_step_all(self._h, C.byref(o), reps), "vmc_sr_step_all")
        return [{k: getattr(r, k) for k, _ in VmcSrReport._fields_} for r in reps]

    def get_sr_matrices(self, shift_rel=0.0, shift_abs=0.0, system=0, with_S=True):
        Np = self.num_params(system)
        S = np.zeros((Np, Np)) if with_S else None
        g = np.zeros(Np)
        _check(self._L.vmc_get_sr_matrices(self._h, system, shift_rel, shift_abs,
                                           _p(S, _F64P) if with_S else None, _p(g, _F64P)),
               "vmc_get_sr_matrices")
        return S, g

    def get_params(self, system=0):
        out = np.zeros(self.num_params(system))
        _check(self._L.vmc_get_params(self._h, system, _p(out, _F64P)), "vmc_get_params")
        return out

    def set_params(self, params, system=0):
        params = np.ascontiguousarray(params, np.float64)
        _check(self._L.vmc_set_params(self._h, system, _p(params, _F64P)), "vmc_set_params")

    # -- check hooks
    def eval_ratios(self, walker, moves, system=0):
        mv = np.ascontiguousarray(moves, np.int32).reshape(-1, 3)
        out = np.zeros(len(mv))
        _check(self._L.vmc_eval_ratios(self._h, system, walker, len(mv), _p(mv, _I32P),
                                       _p(out, _F64P)), "vmc_eval_ratios")
        return out

    def get_inverse(self, walker, system=0):
        N = self.problems[system].Ne // 2
        m = np.zeros((N, N))
        ld = C.c_double()
        sg = C.c_int32()
        _check(self._L.vmc_get_inverse(self._h, system, walker, _p(m, _F64P), C.byref(ld),
                                       C.byref(sg)), "vmc_get_inverse")
        return m, ld.value, sg.value

    def kernel_launches(self):
        return int(self._L.vmc_kernel_launches(self._h))

    def sweep_launch(self):
        """(grid, CTAs per SM, shared-memory bytes) of the sweep kernel (vmc_sweep_launch)."""
        g, o = np.zeros(1, np.int32), np.zeros(1, np.int32)
        b = C.c_int64(0)
        _check(self._L.vmc_sweep_launch(self._h, _p(g, _I32P), _p(o, _I32P), C.byref(b)),
               "vmc_sweep_launch")
        return int(g[0]), int(o[0]), int(b.value)

    def set_projection(self, perm, sign, weight):
        """Quantum-number projection (vmc_set_projection): perm, sign [n_ops, Ns]
        (T_g c^dag_r T_g^-1 = sign[g, r] c^dag_{perm[g, r]}), real weights
        [n_ops]; empty arrays remove it."""
        perm = np.ascontiguousarray(perm, np.int32)
        sign = np.ascontiguousarray(sign, np.int8)
        weight = np.ascontiguousarray(weight, np.float64)
        _check(self._L.vmc_set_projection(self._h, int(weight.size), _p(perm, _I32P),
                                          _p(sign, _I8P), _p(weight, _F64P)),
               "vmc_set_projection")

    def lanczos_moments(self, system=0):
        """First-step power-Lanczos (vmc_lanczos_moments): per-walker F(x, H),
        F(x, H^2) of the current configurations and the moments
        {h1, h2_11, h2_20, h3_12} (walker means)."""
        W = self.n_walkers
        f1, f2, h = np.zeros(W), np.zeros(W), np.zeros(4)
        _check(self._L.vmc_lanczos_moments(self._h, system, _p(f1, _F64P), _p(f2, _F64P),
                                           _p(h, _F64P)), "vmc_lanczos_moments")
        return f1, f2, dict(h1=h[0], h2_11=h[1], h2_20=h[2], h3_12=h[3])

    def test_stall(self, target, system=0, walker=0):
        """Failure-detection test hook (vmc_test_stall): arm one bounded wait
        that cannot complete in the next vmc_sample (STALL_SAMPLE, `walker`)
        or dense S build (STALL_S_BUILD); STALL_NONE disarms."""
        _check(self._L.vmc_test_stall(self._h, int(target), int(system), int(walker)),
               "vmc_test_stall")

    # -- delayed updates
    def set_delay(self, k):
        _check(self._L.vmc_set_delay(self._h, int(k)), "vmc_set_delay")

    def get_delay(self):
        return int(self._L.vmc_get_delay(self._h))

    def tune_delay(self, sweeps=2, candidates=None):
        """Time vmc_sample(0, 1, sweeps) (sweeps + one measurement) per
        candidate depth, keep the fastest.  Returns (chosen, {k: ms per sweep,
        or None where it does not fit})."""
        cand = np.ascontiguousarray(candidates if candidates is not None else (1, 4, 8, 16, 32),
                                    np.int32)
        ms = np.zeros(cand.size)
        chosen = np.zeros(1, np.int32)
        _check(self._L.vmc_tune_delay(self._h, int(sweeps), _p(cand, _I32P), cand.size,
                                      _p(chosen, _I32P), _p(ms, _F64P)), "vmc_tune_delay")
        return int(chosen[0]), {int(k): (float(t) if t >= 0 else None) for k, t in zip(cand, ms)}

    # -- proposals formed together by the sweep
    def set_proposal_batch(self, b):
        _check(self._L.vmc_set_proposal_batch(self._h, int(b)), "vmc_set_proposal_batch")

    def get_proposal_batch(self):
        return int(self._L.vmc_get_proposal_batch(self._h))

    def tune_proposal_batch(self, sweeps=2, candidates=None):
        """Time vmc_sample(sweeps, 0, 0) (sweeps only) per candidate batch
        depth, keep the fastest.  Returns (chosen, {b: ms per sweep})."""
        cand = np.ascontiguousarray(candidates if candidates is not None else (1, 2, 4, 8),
                                    np.int32)
        ms = np.zeros(cand.size)
        chosen = np.zeros(1, np.int32)
        _check(self._L.vmc_tune_proposal_batch(self._h, int(sweeps), _p(cand, _I32P), cand.size,
                                               _p(chosen, _I32P), _p(ms, _F64P)),
               "vmc_tune_proposal_batch")
        return int(chosen[0]), {int(k): float(t) for k, t in zip(cand, ms)}

    def enable_timing(self, on=True):
        _check(self._L.vmc_enable_timing(self._h, 1 if on else 0), "vmc_enable_timing")

    def kernel_times(self):
        """{'sweep'|'init'|'sr'|'sr_gemm': (milliseconds, launches)} since the last call."""
        ms = np.zeros(4)
        cnt = np.zeros(4, np.int64)
        _check(self._L.vmc_kernel_times(self._h, _p(ms, _F64P), cnt.ctypes.data_as(C.POINTER(C.c_int64))),
               "vmc_kernel_times")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(("sweep", "init", "sr", "sr_gemm"))}


def lanczos_alpha(moments):
    """alpha_1 and E_1(alpha_1) of Sec. 3.4 from the moments (vmc_lanczos_alpha)."""
    L = load()
    h = np.array([moments["h1"], moments["h2_11"], moments["h2_20"], moments["h3_12"]])
    a, e = C.c_double(), C.c_double()
    _check(L.vmc_lanczos_alpha(_p(h, _F64P), C.byref(a), C.byref(e)), "vmc_lanczos_alpha")
    return a.value, e.value
