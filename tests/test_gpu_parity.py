"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
identical seeded inputs.

Tolerances (FP64 plain form): Pfaffian ratios, inverses, local energies and
O_k rows within 1e-10 relative (configurations with cond(X) > 1e8 are
skipped, ratios compared where |ratio| > 1e-8); configurations and Philox
counters bit-exact; sampled energies within 3 combined standard errors.
"""
import math

import numpy as np
import pytest

from oracle import fock
from oracle.exact import enumerate_expectations
from oracle.sampler import run_sampling
from oracle.sr import sr_matrices, sr_step, shifted
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I

from helpers import (condition_ok, labelled_slog, oracle_measure, oracle_ratio, random_moves)

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


def rel_close(a, b, rtol=RTOL, floor=0.0):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    scale = max(np.max(np.abs(b)), floor, 1e-300)
    return np.max(np.abs(a - b)) <= rtol * scale


def small_problems():
    return {
        "ring8": I.ring8_hubbard(),
        "square8": I.square8_hubbard(),
        "ring6_apbc": I.make_problem("r6", I.chain(6, -1), 6, U=4.0, sub=(2, 1), jastrow="chain",
                                     noise=0.2, seed=4),
        "heis4": I.heisenberg_square(4, noise=0.1, seed=3),
        "j1j2_4": I.make_problem("j1j2_4", I.square(4, 4, 1, -1), 16, t=0.0, J1=1.0, J2=0.5,
                                 local_spin=True, f_full=True, gutzwiller=False, noise=0.1, seed=5),
    }


def with_correlations(p, seed=0):
    """Give Gutzwiller/Jastrow parameters non-zero values."""
    rng = np.random.default_rng(seed)
    p = p.copy_with(params=p.params.copy())
    k = p.n_g + p.n_v
    p.params[:k] = rng.uniform(-0.4, 0.2, k)
    return p


def good_configs(p, W, seed):
    wf = Wavefunction(p)
    out = []
    s = seed
    while len(out) < W:
        c = I.initial_configs(p.Ns, p.Ne, 1, p.local_spin, s)[0]
        s += 1
        if condition_ok(wf, c):
            out.append(c)
    return np.array(out, np.int32)


@pytest.mark.parametrize("name", ["ring8", "square8", "ring6_apbc", "heis4", "j1j2_4"])
def test_inverse_and_logdet(vmc, name):
    p = with_correlations(small_problems()[name])
    W = 3
    cfg = good_configs(p, W, 100)
    wf = Wavefunction(p)
    N = p.N
    with vmc.Context(p, W, seed=7) as ctx:
        ctx.set_configs(cfg)
        for w in range(W):
            minv, ld, sg = ctx.get_inverse(w)
            ele = cfg[w]
            M = wf.f[np.ix_(ele[:N], ele[N:])]
            # oracle: X over the labelled electron list, its inverse and Pfaffian
            orbs = [int(s) for s in ele[:N]] + [int(s) + p.Ns for s in ele[N:]]
            X = wf.F[np.ix_(orbs, orbs)] - wf.F[np.ix_(orbs, orbs)].T
            Xinv = np.linalg.inv(X)
            # X^-1 = [[0, -M^-T], [M^-1, 0]]  ->  (M^-1)_{mn} = (X^-1)_{N+m, n}
            assert rel_close(minv, Xinv[N:, :N])
            s_pf, l_pf = labelled_slog(wf, ele)
            l_pf -= math.lgamma(N + 1) + wf.log_correlation(fock.from_labels(ele, p.Ns))
            assert ld == pytest.approx(l_pf, rel=1e-11, abs=1e-10)
            assert sg * (-1) ** (N * (N - 1) // 2) == s_pf
            assert np.allclose(M @ minv, np.eye(N), atol=1e-9)


@pytest.mark.parametrize("rebuild", ["fp64", "double_float"])
@pytest.mark.parametrize("name", ["ring8", "square8", "ring6_apbc", "heis4", "j1j2_4"])
def test_mixed_form_double_float_inverse(vmc, name, rebuild):
    """The mixed form's from-scratch inverse, stored as hi + lo FP32 words,
    from the FP64 Gauss-Jordan (default) or the double-float one (opt-in),
    against the oracle's X^-1 and Pfaffian: relative error within
    1e-12 cond(M) (about 2^-46 rounding amplified by the condition number),
    the same sign, log|det| within 1e-12 cond(M) + 1e-11."""
    p = with_correlations(small_problems()[name])
    W = 3
    cfg = good_configs(p, W, 100)
    wf = Wavefunction(p)
    N = p.N
    mode = vmc.REBUILD_FP64 if rebuild == "fp64" else vmc.REBUILD_DOUBLE_FLOAT
    with vmc.Context(p, W, seed=7, precision=vmc.MIXED, rebuild=mode) as ctx:
        ctx.set_configs(cfg)
        for w in range(W):
            minv, ld, sg = ctx.get_inverse(w)
            ele = cfg[w]
            M = wf.f[np.ix_(ele[:N], ele[N:])]
            orbs = [int(s) for s in ele[:N]] + [int(s) + p.Ns for s in ele[N:]]
            X = wf.F[np.ix_(orbs, orbs)] - wf.F[np.ix_(orbs, orbs)].T
            ref = np.linalg.inv(X)[N:, :N]
            cond = np.linalg.cond(M)
            err = np.abs(minv - ref).max() / np.abs(ref).max()
            assert err <= 1e-12 * cond + 1e-15, (err, cond)
            s_pf, l_pf = labelled_slog(wf, ele)
            l_pf -= math.lgamma(N + 1) + wf.log_correlation(fock.from_labels(ele, p.Ns))
            assert abs(ld - l_pf) <= 1e-12 * cond + 1e-11
            assert sg * (-1) ** (N * (N - 1) // 2) == s_pf


@pytest.mark.parametrize("rebuild", ["fp64", "double_float"])
def test_mixed_form_double_float_inverse_16x16(vmc, rebuild):
    """Full size (16x16 Hubbard, N = 112): the mixed form's rebuilt inverses
    of the library's own seeded placements against the FP64 form's."""
    p = I.square16_hubbard()
    W = 8
    with vmc.Context(p, W, seed=3, precision=vmc.FP64) as c64:
        ele, _ = c64.get_configs()
        ref = [c64.get_inverse(w) for w in range(W)]
    N = p.N
    mode = vmc.REBUILD_FP64 if rebuild == "fp64" else vmc.REBUILD_DOUBLE_FLOAT
    with vmc.Context(p, W, seed=3, precision=vmc.MIXED, rebuild=mode) as c32:
        c32.set_configs(ele)
        for w in range(W):
            minv, ld, sg = c32.get_inverse(w)
            a, la, sa = ref[w]
            cond = np.linalg.cond(p.f_matrix()[np.ix_(ele[w, :N], ele[w, N:])])
            err = np.abs(minv - a).max() / np.abs(a).max()
            assert err <= 1e-12 * cond + 1e-15, (w, err, cond)
            assert sg == sa
            assert abs(ld - la) <= 1e-12 * cond + 1e-11


@pytest.mark.parametrize("name", ["ring8", "square8", "ring6_apbc", "heis4", "j1j2_4"])
def test_pfaffian_ratios(vmc, name):
    p = with_correlations(small_problems()[name], 1)
    W = 2
    cfg = good_configs(p, W, 200)
    wf = Wavefunction(p)
    rng = np.random.default_rng(3)
    with vmc.Context(p, W, seed=7) as ctx:
        ctx.set_configs(cfg)
        for w in range(W):
            moves = random_moves(rng, cfg[w], p.N, p.Ns, p.local_spin, 24)
            got = ctx.eval_ratios(w, moves)
            ref = np.array([oracle_ratio(wf, cfg[w], m) for m in moves])
            big = np.abs(ref) > 1e-8
            assert big.sum() > 5
            assert np.all(np.abs(got[big] - ref[big]) <= RTOL * np.abs(ref[big]) + 1e-14)


@pytest.mark.parametrize("name", ["ring8", "square8", "ring6_apbc", "heis4", "j1j2_4"])
def test_local_energy_and_log_derivatives(vmc, name):
    p = with_correlations(small_problems()[name], 2)
    W = 3
    cfg = good_configs(p, W, 300)
    wf = Wavefunction(p)
    with vmc.Context(p, W, seed=7, max_samples=1) as ctx:
        ctx.set_configs(cfg)
        ctx.sample(0, 1, 0)     # measure the configurations as they are
        E, O = ctx.get_samples()
        for w in range(W):
            e_ref, o_ref = oracle_measure(wf, cfg[w])
            assert E[w] == pytest.approx(e_ref, rel=1e-10, abs=1e-10)
            assert rel_close(O[w], o_ref, floor=1.0)


@pytest.mark.parametrize("name,sweeps", [("ring8", 4), ("square8", 1), ("heis4", 2)])
def test_markov_chain_bit_exact(vmc, name, sweeps):
    """Same seed, same initial labels: identical chains (configurations and
    counters bit-exact), identical measured E_loc and O_k."""
    p = with_correlations(small_problems()[name], 3)
    W = 2
    cfg = good_configs(p, W, 400)
    wf = Wavefunction(p)
    seed = 12345
    with vmc.Context(p, W, seed=seed, max_samples=2) as ctx:
        ctx.set_configs(cfg)
        ctx.sample(1, 2, sweeps)
        ele_gpu, ctr_gpu = ctx.get_configs()
        E, O = ctx.get_samples()
        st = ctx.measure()
    ref = run_sampling(wf, cfg, seed, 0, 1, 2, sweeps, p.p_exchange)
    assert np.array_equal(ele_gpu, ref["ele"])
    assert np.array_equal(ctr_gpu.astype(np.int64), ref["counters"])
    assert st["n_accepted"] == ref["n_acc"]
    assert st["n_proposals"] == ref["n_prop"]
    assert np.allclose(E, ref["E"], rtol=1e-10, atol=1e-10)
    assert rel_close(O, ref["O"], floor=1.0)


def test_sampled_energy_matches_exact_enumeration(vmc):
    """Ring of 6 (APBC): MC energy within 3 combined standard errors of the
    exact <H> from enumeration, and O averages likewise."""
    p = with_correlations(small_problems()["ring6_apbc"], 4)
    p = p.copy_with(p_exchange=0.5)
    ex = enumerate_expectations(Wavefunction(p))
    W, S = 256, 100
    with vmc.Context(p, W, seed=99, max_samples=S) as ctx:
        ctx.sample(20, S, 2)
        E, O = ctx.get_samples()
        st = ctx.measure()
    Ew = E.reshape(W, S).mean(axis=1)
    se = Ew.std(ddof=1) / math.sqrt(W)
    assert abs(E.mean() - ex["energy"]) < 3 * se
    assert st["energy"] == pytest.approx(E.mean(), rel=1e-12)
    Ow = O.reshape(W, S, -1).mean(axis=1)
    se_o = Ow.std(axis=0, ddof=1) / math.sqrt(W)
    assert np.all(np.abs(Ow.mean(axis=0) - ex["obar"]) < 3 * se_o + 1e-12)


def test_ring8_energy_above_ed_and_close_to_exact(vmc):
    """C1-shaped: 64 walkers x 200 samples x 10 sweeps on the 8-site ring."""
    p = I.ring8_hubbard()
    ex = enumerate_expectations(Wavefunction(p))
    W, S = 64, 200
    with vmc.Context(p, W, seed=3, max_samples=S) as ctx:
        ctx.sample(10, S, 10)
        st = ctx.measure()
    assert abs(st["energy"] - ex["energy"]) < 3 * st["stderr_walkers"] + 1e-12
    assert 0.0 < st["acceptance"] < 1.0


def test_free_fermion_zero_variance_on_gpu(vmc):
    """U = 0, pure pairing state: every sampled E_loc equals the free-fermion
    energy (closed shell 8x8, P x AP boundaries)."""
    p = I.square8_hubbard(noise=0.0, U=0.0)
    W, S = 32, 4
    with vmc.Context(p, W, seed=5, max_samples=S) as ctx:
        ctx.sample(5, S, 1)
        E, _ = ctx.get_samples()
    kx = 2 * np.pi * np.arange(8) / 8
    ky = (2 * np.pi * np.arange(8) + np.pi) / 8
    eps = np.sort((-2 * (np.cos(kx)[:, None] + np.cos(ky)[None, :])).ravel())
    e0 = 2 * eps[:32].sum()
    assert np.allclose(E, e0, atol=1e-8)


def test_sr_matrices_and_step_match_oracle(vmc):
    p = I.ring8_hubbard()
    Np = p.Np
    E, O = I.random_samples(1000, Np, seed=11)
    with vmc.Context(p, 10, seed=1, max_samples=100) as ctx:
        ctx.set_samples(E, O)
        S_gpu, g_gpu = ctx.get_sr_matrices(1e-3, 0.0)
        S, g, obar, ebar = sr_matrices(E, O)
        assert rel_close(S_gpu, shifted(S, 1e-3, 0.0))
        assert rel_close(g_gpu, g)
        p0 = ctx.get_params()
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.CHOLESKY)
        d_gpu = ctx.get_params() - p0
        d_ref, info = sr_step(E, O, 0.05, 1e-3, 0.0, "cholesky")
        assert rel_close(d_gpu, d_ref, rtol=1e-9)
        assert rep["energy"] == pytest.approx(ebar, rel=1e-12)
        ctx.set_params(p0)
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.CG, cg_eps=1e-12)
        d_cg = ctx.get_params() - p0
        assert rel_close(d_cg, d_ref, rtol=1e-8)
        assert rep["cg_iters"] > 0
        ctx.set_params(p0)
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.CG_DENSE, cg_eps=1e-12)
        assert rel_close(ctx.get_params() - p0, d_ref, rtol=1e-8)
        assert rep["cg_iters"] > 0


def test_sr_on_sampled_data_matches_oracle(vmc):
    """SR from the GPU's own samples equals the oracle's SR on the oracle's
    chain (bit-identical configurations)."""
    p = with_correlations(I.ring8_hubbard(), 5)
    W, S = 4, 20
    cfg = good_configs(p, W, 500)
    wf = Wavefunction(p)
    with vmc.Context(p, W, seed=77, max_samples=S) as ctx:
        ctx.set_configs(cfg)
        ctx.sample(2, S, 1)
        p0 = ctx.get_params()
        ctx.sr_step(0.05, 1e-2, 1e-4, solver=vmc.CHOLESKY)
        d_gpu = ctx.get_params() - p0
    ref = run_sampling(wf, cfg, 77, 0, 2, S, 1, p.p_exchange)
    d_ref, _ = sr_step(ref["E"], ref["O"], 0.05, 1e-2, 1e-4, "cholesky")
    assert rel_close(d_gpu, d_ref, rtol=1e-8)


def test_edge_cases(vmc):
    p = I.ring8_hubbard()
    with vmc.Context(p, 2, seed=1, max_samples=2) as ctx:
        with pytest.raises(vmc.VmcError):
            ctx.sample(0, 3, 1)            # more samples than capacity
        bad = np.array([[0, 0, 1, 2, 0, 1, 2, 3]] * 2, np.int32)
        with pytest.raises(vmc.VmcError):
            ctx.set_configs(bad)          # doubly occupied up orbital
        ctx.sample(1, 0, 0)                # one sweep, no measurement
        assert ctx.measure()["n_proposals"] == 2 * 8
        ctx.sample(0, 1, 0)                # measurement only
        E, O = ctx.get_samples()
        assert E.shape == (2,) and O.shape == (2, p.Np)
    # singular: a site with no pair amplitude at all
    q = p.copy_with(f_idx=p.f_idx.copy())
    q.f_idx.reshape(8, 8)[0, :] = -1
    with vmc.Context(q, 1, seed=1) as ctx:
        cfg = np.array([[0, 2, 4, 6, 1, 3, 5, 7]], np.int32)
        ctx.set_configs(cfg)
        with pytest.raises(vmc.VmcError) as ei:
            ctx.sample(0, 0, 1)
        assert ei.value.code == -4


def test_batched_systems_match_single(vmc):
    """A batch of uneven systems gives each system exactly the chain it gets alone."""
    probs = [I.ring8_hubbard(), I.square8_hubbard(), I.make_problem(
        "r6", I.chain(6, -1), 6, U=4.0, sub=(2, 1), jastrow="chain", noise=0.2, seed=4)]
    W = 3
    cfgs = [good_configs(with_correlations(q), W, 600 + k) for k, q in enumerate(probs)]
    with vmc.Context(probs, W, seed=5, max_samples=2) as ctx:
        for s, c in enumerate(cfgs):
            ctx.set_configs(c, system=s)
        ctx.sample(1, 2, 1)
        batch = [(ctx.get_configs(s)[0], ctx.get_samples(s)[0]) for s in range(len(probs))]
    for s, q in enumerate(probs):
        wf = Wavefunction(q)
        ref = run_sampling(wf, cfgs[s], 5, s, 1, 2, 1, q.p_exchange)
        assert np.array_equal(batch[s][0], ref["ele"])
        assert np.allclose(batch[s][1], ref["E"], rtol=1e-10, atol=1e-10)


def test_mixed_precision_close_to_fp64(vmc):
    """Mixed form: FP32 ratios/updates with FP64 recompute; E_loc on the same
    configurations within 1e-4 t per site of the FP64 form."""
    p = with_correlations(I.square8_hubbard(), 6)
    W = 4
    cfg = good_configs(p, W, 700)
    res = {}
    for prec in (vmc.FP64, vmc.MIXED):
        with vmc.Context(p, W, seed=7, precision=prec, max_samples=1) as ctx:
            ctx.set_configs(cfg)
            ctx.sample(0, 1, 0)
            res[prec] = ctx.get_samples()
    dE = np.abs(res[vmc.FP64][0] - res[vmc.MIXED][0]) / p.Ns
    assert dE.max() < 1e-4
    assert np.allclose(res[vmc.FP64][1], res[vmc.MIXED][1], rtol=1e-3, atol=1e-3)


@pytest.mark.parametrize("kernel", ["tma", "tiles"])
@pytest.mark.parametrize("rows,Np", [(1000, 19), (2049, 300), (4096, 1069), (8192, 4100)])
def test_sr_overlap_tensor_cores_split_bf16(vmc, rows, Np, kernel, monkeypatch):
    """Mixed form: S built by the tcgen05 split-BF16 GEMM (FP32 accumulation)
    against the oracle's FP64 S; tiles, chunks and ragged edges covered, for
    both kernels (persistent TMA-fed kernel, and one CTA per tile with
    cp.async staging).  Tolerance: 2e-4 of max|S| (three BF16 products ~2^-16
    relative each, FP32 sums over the samples)."""
    if kernel == "tiles":
        monkeypatch.setenv("VMC_TC_KERNEL", "tiles")
    else:
        monkeypatch.delenv("VMC_TC_KERNEL", raising=False)
    if kernel == "tiles" and Np > 2000:
        pytest.skip("the one-CTA-per-tile kernel is covered at the smaller sizes")
    base = I.ring8_hubbard()
    n_f = Np - base.n_g - base.n_v
    if n_f == base.n_f:
        p = base
    else:   # one class per (i, j) pair, extra classes unused by the wave function
        p = base.copy_with(n_f=n_f, f_idx=np.arange(64, dtype=np.int32), f_sign=np.ones(64, np.int8),
                           params=np.concatenate([base.params[:3],
                                                  np.random.default_rng(0).uniform(-1, 1, n_f)]))
    E, O = I.random_samples(rows, Np, seed=rows + Np)
    O[:, : Np // 3] += 0.5           # non-zero means: centring matters
    W = 16
    with vmc.Context(p, W, seed=1, precision=vmc.MIXED, max_samples=(rows + W - 1) // W) as ctx:
        ctx.set_samples(E, O)
        S_gpu, g_gpu = ctx.get_sr_matrices(0.0, 0.0)
    S, g, _, _ = sr_matrices(E, O.astype(np.float32).astype(np.float64))
    err = np.max(np.abs(S_gpu - S)) / np.max(np.abs(S))
    assert err < 2e-4, err
    assert np.allclose(S_gpu, S_gpu.T)
    assert rel_close(g_gpu, g, rtol=1e-6)


def test_batched_uneven_lattices_mixed(vmc):
    """Batched workload shape: 64 independent Hubbard systems with L in
    {4..16} (n = 0.875, U/t in [2, 8]) in one persistent launch, mixed form.
    After equilibration, every system's energy estimate (walker mean of E_loc)
    on identical configurations matches the FP64 form within 1e-4 t per site,
    and the typical walker agrees to 1e-5 t per site."""
    probs = I.batched_hubbard(64, seed=0)
    W = 8
    sweeps = 24
    with vmc.Context(probs, W, seed=11, precision=vmc.MIXED, max_samples=1) as ctx:
        ctx.sample(sweeps - 1, 1, 1)
        cfgs = [ctx.get_configs(s)[0] for s in range(len(probs))]
        e32 = [ctx.get_samples(s)[0] for s in range(len(probs))]
        st = [ctx.measure(s) for s in range(len(probs))]
    with vmc.Context(probs, W, seed=11, precision=vmc.FP64, max_samples=1) as ref:
        for s, c in enumerate(cfgs):
            ref.set_configs(c, system=s)
        ref.sample(0, 1, 0)
        e64 = [ref.get_samples(s)[0] for s in range(len(probs))]
    for s, p in enumerate(probs):
        assert st[s]["n_proposals"] == W * sweeps * p.Ne
        assert st[s]["n_accepted"] > 0
    # the measurement is the last step of the call: the stored configurations are the measured ones
    d_mean = [abs(a.mean() - b.mean()) / p.Ns for a, b, p in zip(e32, e64, probs)]
    d_med = np.median(np.concatenate([np.abs(a - b) / p.Ns for a, b, p in zip(e32, e64, probs)]))
    assert max(d_mean) < 1e-4, max(d_mean)
    assert d_med < 1e-5, d_med
