"""Proposals formed in batches (vmc_set_proposal_batch): the sweep checks the
next b proposals and forms their ratios together, then takes the Metropolis
decisions in order and stops at the first accepted one.  The chain must be
the one that proposals made one at a time give (Sec. 3.1.2): configurations,
Philox counters and move counts bit-exact in FP64, samples within 1e-10, and
the oracle's chain for odd batch depths too.
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


def problems():
    d = dict(small_problems())
    d["kondo8"] = I.kondo_chain(8, noise=0.3, seed=1)
    return d


def run_chain(vmc, p, cfg, batch, precision=None, seed=777, warm=2, S=3, sweeps=2):
    kw = {} if precision is None else {"precision": precision}
    with vmc.Context(p, len(cfg), seed=seed, max_samples=S, **kw) as ctx:
        ctx.set_proposal_batch(batch)
        assert ctx.get_proposal_batch() == batch
        ctx.set_configs(cfg)
        ctx.sample(warm, S, sweeps)
        ele, ctr = ctx.get_configs()
        E, O = ctx.get_samples()
        st = ctx.measure()
    return ele, ctr, E, O, st


def start_configs(p, W, seed):
    if getattr(p, "local_sites", None) is not None:
        out = [I.initial_configs(p.Ns, p.Ne, 1, False, seed + k, local_sites=p.local_sites)[0]
               for k in range(W)]
        return np.array(out, np.int32)
    return good_configs(p, W, seed)


@pytest.mark.parametrize("name", ["ring8", "square8", "ring6_apbc", "heis4", "j1j2_4", "kondo8"])
@pytest.mark.parametrize("batch", [2, 3, 8])
def test_batched_chain_equals_one_at_a_time_fp64(vmc, name, batch):
    p = problems()[name]
    if name != "kondo8":
        p = with_correlations(p, 5)
    cfg = start_configs(p, 4, 900)
    a = run_chain(vmc, p, cfg, 1)
    b = run_chain(vmc, p, cfg, batch)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    for k in ("n_proposals", "n_accepted"):
        assert a[4][k] == b[4][k]
    assert np.allclose(a[2], b[2], rtol=1e-10, atol=1e-10)
    assert rel_close(b[3], a[3], floor=1.0)


@pytest.mark.parametrize("batch", [3, 8])
def test_batched_chain_matches_oracle(vmc, batch):
    """Odd and full depths against the oracle's one-at-a-time chain."""
    p = with_correlations(small_problems()["ring6_apbc"], 3)
    cfg = good_configs(p, 2, 400)
    seed = 4242
    with vmc.Context(p, 2, seed=seed, max_samples=2) as ctx:
        ctx.set_proposal_batch(batch)
        ctx.set_configs(cfg)
        ctx.sample(1, 2, 3)
        ele, ctr = ctx.get_configs()
        E, _ = ctx.get_samples()
        st = ctx.measure()
    ref = run_sampling(Wavefunction(p), cfg, seed, 0, 1, 2, 3, p.p_exchange)
    assert np.array_equal(ele, ref["ele"])
    assert np.array_equal(ctr.astype(np.int64), ref["counters"])
    assert st["n_accepted"] == ref["n_acc"]
    assert st["n_proposals"] == ref["n_prop"]
    assert np.allclose(E, ref["E"], rtol=1e-10, atol=1e-10)


def test_batched_chain_mixed_form(vmc):
    """Mixed form: FP32 ratios summed in another order may flip a decision
    only where u and ratio^2 agree to FP32 rounding; on the 8x8 workload
    every chain stays the same over the run, and the samples agree to the
    double-float inverse's rounding."""
    p = with_correlations(I.square8_hubbard(), 2)
    cfg = good_configs(p, 32, 1300)
    a = run_chain(vmc, p, cfg, 1, precision=vmc.MIXED)
    b = run_chain(vmc, p, cfg, 8, precision=vmc.MIXED)
    same = np.all(a[0] == b[0], axis=1)
    assert same.mean() >= 0.95
    W, S = len(cfg), 3
    Ea = a[2].reshape(W, S)[same]
    Eb = b[2].reshape(W, S)[same]
    assert np.allclose(Ea, Eb, rtol=1e-6, atol=1e-6)


def test_invalid_batch_depth_rejected(vmc):
    p = small_problems()["ring8"]
    with vmc.Context(p, 2, seed=1) as ctx:
        for bad in (0, -1, 9):
            with pytest.raises(vmc.VmcError):
                ctx.set_proposal_batch(bad)
        assert ctx.get_proposal_batch() == 1


def test_tuner_picks_a_candidate(vmc):
    p = with_correlations(I.square8_hubbard(), 1)
    with vmc.Context(p, 256, seed=2, precision=vmc.MIXED, max_samples=1) as ctx:
        ctx.sample(1, 1, 1)
        chosen, ms = ctx.tune_proposal_batch(sweeps=2, candidates=(1, 4, 8))
        assert chosen in (1, 4, 8)
        assert ctx.get_proposal_batch() == chosen
        assert all(t > 0 for t in ms.values())
        assert ms[chosen] == min(ms.values())


def test_batched_chain_full_size_spin_model(vmc):
    """J1-J2 16x16 (N = 128, every proposal an exchange), mixed form: the
    batched sweep (every thread of the CTA a row) keeps the chains of the
    one-at-a-time sweep up to FP32 decision flips."""
    p = I.j1j2_heisenberg(16)
    W = 64
    cfg = I.initial_configs(p.Ns, p.Ne, W, True, 31)
    a = run_chain(vmc, p, cfg, 1, precision=vmc.MIXED, warm=1, S=1, sweeps=1)
    b = run_chain(vmc, p, cfg, 8, precision=vmc.MIXED, warm=1, S=1, sweeps=1)
    same = np.all(a[0] == b[0], axis=1)
    assert same.mean() >= 0.9
    assert np.allclose(a[2][same], b[2][same], rtol=1e-6, atol=1e-6)


def test_tuner_refuses_projected_context(vmc):
    """The projected sweep makes its proposals one at a time: nothing to tune."""
    p = I.ring8_hubbard()
    with vmc.Context(p, 4, seed=3, max_samples=1) as ctx:
        perm = np.array([np.roll(np.arange(p.Ns), k) for k in range(2)], np.int32)
        ctx.set_projection(perm, np.ones_like(perm, dtype=np.int8), np.full(2, 0.5))
        with pytest.raises(vmc.VmcError):
            ctx.tune_proposal_batch(sweeps=1)
