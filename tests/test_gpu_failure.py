"""Failure detection on the GPU without a GPU fault: the bounded device waits.

vmc_test_stall arms one wait that cannot complete (an mbarrier on which no
copy or MMA was issued), polled a bounded number of times; the kernel gives
up with nothing in flight and the call returns VMC_ETIMEOUT.  The context
stays usable: the skipped walker and every other walker continue their
Markov chains exactly as the oracle's chains do, and the failed SR step
leaves the parameters unchanged, after which the next step solves the
complete S~ of the same samples.
"""
import numpy as np
import pytest

from oracle.sampler import run_sampling
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I

from helpers import condition_ok

pytestmark = pytest.mark.gpu

ETIMEOUT = -6


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


def configs(p, W, seed):
    wf = Wavefunction(p)
    out, s = [], seed
    while len(out) < W:
        c = I.initial_configs(p.Ns, p.Ne, 1, p.local_spin, s)[0]
        s += 1
        if condition_ok(wf, c):
            out.append(c)
    return np.array(out, np.int32)


def oracle_call(wf, ele, ctr, p, walkers):
    """One vmc_sample(1, 2, 1) by the oracle, every walker on its own Philox
    stream (walker index = row); the rows of `walkers` are returned."""
    ref = run_sampling(wf, ele, 31, 0, 1, 2, 1, p.p_exchange, counters=ctr)
    W = len(ele)
    return (ref["ele"][walkers], ref["counters"][walkers],
            ref["E"].reshape(W, 2)[walkers].ravel())


def test_sample_timeout_skips_one_walker_and_the_chains_continue(vmc):
    p = I.ring8_hubbard()
    wf = Wavefunction(p)
    W, stalled = 4, 2
    cfg = configs(p, W, 5)
    ctr0 = np.zeros(W, np.int64)
    others = [w for w in range(W) if w != stalled]
    with vmc.Context(p, W, seed=31, max_samples=2) as ctx:
        ctx.set_configs(cfg)
        ctx.test_stall(vmc.STALL_SAMPLE, walker=stalled)
        with pytest.raises(vmc.VmcError) as e:
            ctx.sample(1, 2, 1)
        assert e.value.code == ETIMEOUT
        assert ctx.measure()["n_flagged"] >= 1
        ele1, ctr1 = ctx.get_configs()
        # the skipped walker did not move; the others made one call's sweeps
        assert np.array_equal(ele1[stalled], cfg[stalled]) and ctr1[stalled] == 0
        ref_e, ref_c, _ = oracle_call(wf, cfg, ctr0, p, others)
        assert np.array_equal(ele1[others], ref_e)
        assert np.array_equal(ctr1[others].astype(np.int64), ref_c)
        # the hook is one-shot: the next call samples every walker
        ctx.sample(1, 2, 1)
        ele2, ctr2 = ctx.get_configs()
        E2, _ = ctx.get_samples()
        assert ctx.measure()["n_flagged"] == 0
    ref_s = oracle_call(wf, cfg, ctr0, p, [stalled])
    ref_o = oracle_call(wf, ele1, ctr1.astype(np.int64), p, others)
    assert np.array_equal(ele2[stalled], ref_s[0][0]) and ctr2[stalled] == ref_s[1][0]
    assert np.array_equal(ele2[others], ref_o[0])
    assert np.array_equal(ctr2[others].astype(np.int64), ref_o[1])
    E2 = E2.reshape(W, 2)
    assert np.allclose(E2[stalled], ref_s[2], rtol=1e-10, atol=1e-10)
    assert np.allclose(E2[others].ravel(), ref_o[2], rtol=1e-10, atol=1e-10)


def test_s_build_timeout_leaves_the_parameters_and_the_next_step_is_exact(vmc):
    p = I.ring8_hubbard()
    W = 64
    with vmc.Context(p, W, seed=3, precision=vmc.MIXED, max_samples=4) as ctx:
        ctx.sample(4, 4, 1)
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-12)
        if vmc.S_KERNELS[rep["s_kernel"]] != "tcgen05_tma_persistent":
            pytest.skip("the persistent tensor-core S kernel is not in use on this device")
        ctx.sample(0, 4, 1)
        p0 = ctx.get_params()
        ctx.test_stall(vmc.STALL_S_BUILD)
        with pytest.raises(vmc.VmcError) as e:
            ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-12)
        assert e.value.code == ETIMEOUT
        assert np.array_equal(ctx.get_params(), p0)
        # the next build is complete: S~ and g of the same samples, solved in FP64
        St, g = ctx.get_sr_matrices(1e-3, 0.0)
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-12)
        x = -(ctx.get_params() - p0) / 0.05
    assert rep["fallback"] == 0 and rep["s_kernel"] == 2
    assert np.all(np.isfinite(St)) and np.all(np.diag(St) > 0)
    x_ref = np.linalg.solve(St, g)
    assert np.max(np.abs(x - x_ref)) <= 1e-7 * np.max(np.abs(x_ref))
