"""Parity at the benchmark's full size and launch configuration: the 16x16
Hubbard lattice (U/t = 8, Ne = 224, APBC, Np = 1069), 4096 walkers, four
samples per walker per call, in-sweep FP64 recompute every 256 accepted
moves.

The oracle computes sampled outputs one by one (a local energy at this size
is about a thousand 224 x 224 Parlett-Reid Pfaffians):

* mixed form: E_loc of sampled rows within 1e-4 t per site of the oracle,
  O_k rows within 1e-3 of max(1, |O|) (FP32 inverse entries);
* plain FP64 form: E_loc and O_k of sampled rows within 1e-10;
* SR from the GPU's own 16384 sample rows: g within 1e-10 and the
  split-BF16 tensor-core S~ within 2e-4 of max |S~| of the FP64 product of
  the same rows; the mixed solve's update has FP64 backward error < 1e-3
  against the FP64 S~ (the split-BF16 error of S~ bounds it).
"""
import numpy as np
import pytest

from oracle import fock
from oracle.hamiltonian import local_energy
from oracle.sr import sr_matrices, shifted
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W, S = 4096, 4
CHECK_WALKERS = (0, 2047, 4095)


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


@pytest.fixture(scope="module")
def problem():
    return I.square16_hubbard()


def oracle_rows(p, params, ele_rows):
    wf = Wavefunction(p, params)
    out = []
    for ele in ele_rows:
        n = fock.from_labels(ele, p.Ns)
        out.append((local_energy(wf, n), wf.log_derivatives(n)))
    return out


def run(vmc, p, precision, warm):
    with vmc.Context(p, W, seed=2024, precision=precision, max_samples=S,
                     recompute_every=256 if precision == vmc.MIXED else -1) as ctx:
        ctx.sample(warm, 0, 0)
        ctx.sample(0, S, 1)
        E, O = ctx.get_samples()
        ele, _ = ctx.get_configs()
        params = ctx.get_params()
        st = ctx.measure()
        St, g = ctx.get_sr_matrices(1e-3, 0.0)
        p0 = params.copy()
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-12)
        x = -(ctx.get_params() - p0) / 0.05
    return dict(E=E, O=O, ele=ele, params=params, st=st, St=St, g=g, x=x, rep=rep)


@pytest.fixture(scope="module")
def mixed(vmc, problem):
    return run(vmc, problem, vmc.MIXED, 10)


def test_fullsize_mixed_sampled_rows_match_oracle(problem, mixed):
    p = problem
    assert mixed["st"]["n_proposals"] == W * (10 + S) * p.Ne
    # the measurement is the last step of the call: row w*S + S-1 is the stored configuration
    rows = [w * S + S - 1 for w in CHECK_WALKERS]
    ref = oracle_rows(p, mixed["params"], [mixed["ele"][w] for w in CHECK_WALKERS])
    for r, (e_ref, o_ref) in zip(rows, ref):
        assert abs(mixed["E"][r] - e_ref) / p.Ns < 1e-4, (r, mixed["E"][r], e_ref)
        scale = max(1.0, np.max(np.abs(o_ref)))
        assert np.max(np.abs(mixed["O"][r] - o_ref)) < 1e-3 * scale


def test_fullsize_sr_from_own_samples(problem, mixed):
    E, O = mixed["E"], mixed["O"].astype(np.float64)
    S_ref, g_ref, _, _ = sr_matrices(E, O)
    St_ref = shifted(S_ref, 1e-3, 0.0)
    assert np.max(np.abs(mixed["g"] - g_ref)) <= 1e-10 * np.max(np.abs(g_ref))
    assert np.max(np.abs(mixed["St"] - St_ref)) <= 2e-4 * np.max(np.abs(St_ref))
    assert mixed["rep"]["fallback"] == 0
    res = np.linalg.norm(g_ref - St_ref @ mixed["x"]) / np.linalg.norm(g_ref)
    assert res < 1e-3, res


def well_conditioned(p, params, ele_rows, limit=1e8):
    """Walkers whose M has cond < limit (the 1e-10 comparisons exclude the
    rest, as for the small systems)."""
    wf = Wavefunction(p, params)
    N = p.N
    return [k for k, e in enumerate(ele_rows)
            if np.linalg.cond(wf.f[np.ix_(e[:N], e[N:])]) < limit]


def test_fullsize_fp64_sampled_rows_match_oracle(vmc, problem):
    p = problem
    r64 = run(vmc, p, vmc.FP64, 1)
    cand = [w for w in range(0, W, 97)]
    ok = well_conditioned(p, r64["params"], [r64["ele"][w] for w in cand])
    walkers = [cand[k] for k in ok[:2]]
    assert len(walkers) == 2
    rows = [w * S + S - 1 for w in walkers]
    ref = oracle_rows(p, r64["params"], [r64["ele"][w] for w in walkers])
    for r, (e_ref, o_ref) in zip(rows, ref):
        assert r64["E"][r] == pytest.approx(e_ref, rel=1e-10, abs=1e-10)
        scale = max(1.0, np.max(np.abs(o_ref)))
        assert np.max(np.abs(r64["O"][r] - o_ref)) <= 1e-10 * scale


# --- learned part at full lattice size: 16x16 Hubbard x MLP (512 -> 1024 -> 1)

def _mlp_run(vmc, p, precision):
    with vmc.Context(p, 64, seed=77, precision=precision, max_samples=1) as ctx:
        ctx.sample(1, 1, 1)
        E, O = ctx.get_samples()
        ele, _ = ctx.get_configs()
        params = ctx.get_params()
    return E, O, ele, params


def test_fullsize_mlp_sampled_rows_match_oracle(vmc):
    """FP64 form with the MLP factor (Np = 527,406): E_loc and the whole O_k
    row (Gutzwiller, Jastrow, pair orbitals and the MLP gradients) of sampled
    rows within 1e-10 of the oracle; mixed form (BF16 W1) E_loc within
    5e-3 t per site (the BF16 rounding of W1 moves the log-amplitude)."""
    p = I.square16_hubbard_mlp()
    E, O, ele, params = _mlp_run(vmc, p, vmc.FP64)
    ok = well_conditioned(p, params, [ele[w] for w in range(0, 64, 7)])
    walkers = [range(0, 64, 7)[k] for k in ok[:2]]
    assert len(walkers) == 2
    ref = oracle_rows(p, params, [ele[w] for w in walkers])
    for w, (e_ref, o_ref) in zip(walkers, ref):
        assert E[w] == pytest.approx(e_ref, rel=1e-10, abs=1e-10)
        assert np.max(np.abs(O[w] - o_ref)) <= 1e-10 * max(1.0, np.max(np.abs(o_ref)))
    E32, _, ele32, params32 = _mlp_run(vmc, p, vmc.MIXED)
    ref32 = oracle_rows(p, params32, [ele32[w] for w in walkers])
    for w, (e_ref, _) in zip(walkers, ref32):
        assert abs(E32[w] - e_ref) / p.Ns < 5e-3


# --- J1-J2 shape: 16x16 Heisenberg as doublon-free fermions, full f (Np = 65536)

def test_fullsize_j1j2_sampled_rows_match_oracle(vmc):
    """Exchange-only sampling of the 16x16 J1-J2 model (J2/J1 = 0.5): E_loc
    (each exchange term a labelled swap ratio) and the 65,536-entry O_k row
    of sampled rows within 1e-10 of the oracle in FP64; the mixed form's
    E_loc within 1e-4 J per site."""
    p = I.j1j2_heisenberg(16, 0.5)
    rows = {}
    for prec in (vmc.FP64, vmc.MIXED):
        with vmc.Context(p, 64, seed=5, precision=prec, max_samples=1) as ctx:
            ctx.sample(2, 1, 1)
            E, O = ctx.get_samples()
            ele, _ = ctx.get_configs()
            rows[prec] = (E, O, ele, ctx.get_params())
    E, O, ele, params = rows[vmc.FP64]
    cand = list(range(0, 64, 9))
    ok = well_conditioned(p, params, [ele[w] for w in cand])
    walkers = [cand[k] for k in ok[:2]]
    assert len(walkers) == 2
    ref = oracle_rows(p, params, [ele[w] for w in walkers])
    for w, (e_ref, o_ref) in zip(walkers, ref):
        assert E[w] == pytest.approx(e_ref, rel=1e-10, abs=1e-10)
        assert np.max(np.abs(O[w] - o_ref)) <= 1e-10 * max(1.0, np.max(np.abs(o_ref)))
    E32, _, ele32, params32 = rows[vmc.MIXED]
    ref32 = oracle_rows(p, params32, [ele32[w] for w in walkers])
    for w, (e_ref, _) in zip(walkers, ref32):
        assert abs(E32[w] - e_ref) / p.Ns < 1e-4


# --- 8x8 FP64 workload (1024 walkers) and the 64-system uneven batch

def test_fullsize_square8_fp64_sampled_rows_match_oracle(vmc):
    """8x8 Hubbard (P x AP, Ne = 64, U/t = 4), 1024 walkers, FP64 everywhere:
    sampled E_loc and O_k rows within 1e-10 of the oracle."""
    p = I.square8_hubbard()
    with vmc.Context(p, 1024, seed=8, precision=vmc.FP64, max_samples=2) as ctx:
        ctx.sample(2, 2, 1)
        E, O = ctx.get_samples()
        ele, _ = ctx.get_configs()
        params = ctx.get_params()
    cand = [0, 511, 1023, 300]
    ok = well_conditioned(p, params, [ele[w] for w in cand])
    walkers = [cand[k] for k in ok[:3]]
    assert len(walkers) >= 2
    ref = oracle_rows(p, params, [ele[w] for w in walkers])
    for w, (e_ref, o_ref) in zip(walkers, ref):
        r = w * 2 + 1
        assert E[r] == pytest.approx(e_ref, rel=1e-10, abs=1e-10)
        assert np.max(np.abs(O[r] - o_ref)) <= 1e-10 * max(1.0, np.max(np.abs(o_ref)))


def test_fullsize_batch64_mixed_sampled_rows_match_oracle(vmc):
    """64 uneven Hubbard systems in one context (L in {4..16}, n = 0.875,
    U/t in [2, 8]), mixed form with the in-sweep FP64 recompute every 64
    accepted moves: for one system of each size, sampled E_loc within 1e-4 t
    per site of the oracle."""
    probs = I.batched_hubbard(64, seed=0)
    with vmc.Context(probs, 64, seed=11, precision=vmc.MIXED, max_samples=2,
                     recompute_every=64) as ctx:
        ctx.sample(4, 2, 1)
        got = {}
        for s, p in enumerate(probs):
            if p.Ns in got:
                continue
            E, _ = ctx.get_samples(s)
            ele, _ = ctx.get_configs(s)
            got[p.Ns] = (s, E, ele, ctx.get_params(s))
    assert len(got) == 7
    for Ns, (s, E, ele, params) in got.items():
        p = probs[s]
        ok = well_conditioned(p, params, [ele[w] for w in range(4)])
        w = ok[0]
        (e_ref, _), = oracle_rows(p, params, [ele[w]])
        assert abs(E[w * 2 + 1] - e_ref) / Ns < 1e-4, (Ns, E[w * 2 + 1], e_ref)
