"""GPU parity of the delayed inverse updates (fast updates of Sec. 3.1.2
applied k at a time): the current inverse is G0 - sum_i u_i v_i^T, ratios
are corrected by the sum, and the pairs are folded into G0 by one rank-k
product.

Pins: in FP64 the delayed form reproduces the oracle's Markov chain bit for
bit (configurations, counters) with E_loc and O_k within 1e-10; in the mixed
form the stored inverse after sampling matches a fresh FP64 inverse of the
configuration's M, and E_loc on identical configurations matches the FP64
form within 1e-4 t per site.
"""
import numpy as np
import pytest

from oracle.sampler import run_sampling
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I

from test_gpu_parity import good_configs, rel_close, small_problems, with_correlations

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


@pytest.mark.parametrize("k", [2, 5, 32])
@pytest.mark.parametrize("name,sweeps", [("ring8", 4), ("square8", 2), ("ring6_apbc", 6),
                                         ("heis4", 2)])
def test_delayed_fp64_chain_matches_oracle(vmc, name, sweeps, k):
    p = with_correlations(small_problems()[name], 3)
    W = 2
    cfg = good_configs(p, W, 400)
    wf = Wavefunction(p)
    seed = 4242
    with vmc.Context(p, W, seed=seed, max_samples=2, delay_k=k) as ctx:
        assert ctx.get_delay() == k
        ctx.set_configs(cfg)
        ctx.sample(1, 2, sweeps)
        ele_gpu, ctr_gpu = ctx.get_configs()
        E, O = ctx.get_samples()
        st = ctx.measure()
    ref = run_sampling(wf, cfg, seed, 0, 1, 2, sweeps, p.p_exchange)
    assert np.array_equal(ele_gpu, ref["ele"])
    assert np.array_equal(ctr_gpu.astype(np.int64), ref["counters"])
    assert st["n_accepted"] == ref["n_acc"]
    assert np.allclose(E, ref["E"], rtol=1e-10, atol=1e-10)
    assert rel_close(O, ref["O"], floor=1.0)


def _inverse_errors(vmc, p, W, k, sweeps):
    """Per-walker max |Minv_stored - inv(M)| / max |inv(M)| after `sweeps`
    sweeps of the mixed form with delay depth k and no in-sweep recompute."""
    wf = Wavefunction(p)
    N = p.N
    with vmc.Context(p, W, seed=21, precision=vmc.MIXED, max_samples=1, delay_k=k,
                     recompute_every=-1) as ctx:
        ctx.sample(sweeps, 0, 0)
        st = ctx.measure()
        ele, _ = ctx.get_configs()
        err = []
        for w in range(W):
            minv, _, _ = ctx.get_inverse(w)
            ref = np.linalg.inv(wf.f[np.ix_(ele[w, :N], ele[w, N:])])
            err.append(np.max(np.abs(minv - ref)) / np.max(np.abs(ref)))
    return np.array(err), st


@pytest.mark.parametrize("k", [4, 16])
def test_delayed_mixed_inverse_matches_fresh(vmc, k):
    """After sampling with k pending updates the stored inverse of every
    walker matches the FP64 inverse of its M to FP32 rounding (the delayed
    form keeps FP32 words only), and the immediate updates, which keep the
    double-float inverse, are at least as close (here far closer)."""
    p = with_correlations(I.square8_hubbard(), 6)
    W = 16
    e_imm, _ = _inverse_errors(vmc, p, W, 1, 6)
    e_dly, st = _inverse_errors(vmc, p, W, k, 6)
    assert st["n_hop_accepted"] > 4 * W
    assert e_dly.max() < 1e-2, e_dly.max()
    assert np.median(e_imm) <= np.median(e_dly), (np.median(e_imm), np.median(e_dly))
    assert e_imm.max() < 1e-6, e_imm.max()


def _energy_error(vmc, p, W, k):
    """Per-walker |E_mixed - E_fp64| / Ns on the configurations the mixed form
    (delay depth k) reached after a few sweeps."""
    with vmc.Context(p, W, seed=5, precision=vmc.MIXED, max_samples=1, delay_k=k) as ctx:
        ctx.sample(3, 1, 1)
        e32, _ = ctx.get_samples()
        cfg, _ = ctx.get_configs()
        st = ctx.measure()
    with vmc.Context(p, W, seed=5, precision=vmc.FP64, max_samples=1) as ref:
        ref.set_configs(cfg)
        ref.sample(0, 1, 0)
        e64, _ = ref.get_samples()
    assert st["n_hop_accepted"] > 0
    return np.abs(e32 - e64) / p.Ns


@pytest.mark.parametrize("k", [8, 16])
def test_delayed_mixed_energy_matches_fp64_square16(vmc, k):
    """16x16 Hubbard (U/t = 8, Ne = 224) with delayed updates: E_loc on the
    stored configurations within 1e-4 t per site of the FP64 form."""
    d = _energy_error(vmc, I.square16_hubbard(), 8, k)
    assert d.max() < 1e-4, d.max()


def test_delayed_mixed_energy_and_immediate_double_float(vmc):
    """8x8 Hubbard with random Gutzwiller/Jastrow values (some walkers poorly
    conditioned): E_loc against FP64 on the same configurations.  The
    immediate updates (double-float inverse) stay within 1e-5 t per site on
    every walker; the delayed form (FP32 words) at the FP32 level, no better."""
    p = with_correlations(I.square8_hubbard(), 6)
    d1 = _energy_error(vmc, p, 8, 1)
    d8 = _energy_error(vmc, p, 8, 8)
    assert d1.max() < 1e-5, d1.max()
    assert np.median(d1) <= np.median(d8), (np.median(d1), np.median(d8))
    assert np.median(d8) < 1e-3, np.median(d8)


def test_delayed_batched_uneven_systems(vmc):
    """Uneven batch (N from 7 to 112) with delayed updates: identical chains to
    the immediate form in FP64."""
    probs = I.batched_hubbard(8, seed=1)
    W = 2
    res = []
    for k in (0, 8):
        with vmc.Context(probs, W, seed=9, precision=vmc.FP64, max_samples=1, delay_k=k) as ctx:
            ctx.sample(2, 1, 1)
            res.append([(ctx.get_configs(s)[0], ctx.get_samples(s)[0]) for s in range(len(probs))])
    for (c0, e0), (c1, e1) in zip(*res):
        assert np.array_equal(c0, c1)
        assert np.allclose(e0, e1, rtol=1e-10, atol=1e-10)


def test_tune_delay_and_limits(vmc):
    p = I.square8_hubbard()
    with vmc.Context(p, 64, seed=3, precision=vmc.MIXED, max_samples=1) as ctx:
        assert ctx.get_delay() == 0
        chosen, ms = ctx.tune_delay(sweeps=1, candidates=(1, 4, 8))
        assert chosen in (1, 4, 8)
        assert all(t is not None and t > 0 for t in ms.values())
        assert ctx.get_delay() == chosen
        for bad in (-1, 33):
            with pytest.raises(vmc.VmcError):
                ctx.set_delay(bad)
        assert ctx.get_delay() == chosen
        ctx.set_delay(1)
        ctx.sample(0, 1, 1)
        assert np.isfinite(ctx.measure()["energy"])
