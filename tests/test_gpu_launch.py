"""Launch configuration of the sweep kernel on the 16x16 Hubbard workload
(U/t = 8, Ne = 224, N = 112): in the mixed form one walker's shared-memory
block (the double-float M^-1, two FP32 words per entry, and the walker's
vectors and tables) must leave room for two CTAs per SM, so that the
persistent grid has two walkers in flight on every SM."""
import pytest

from paper_1711_11418_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


def test_mixed_16x16_runs_two_walkers_per_sm(vmc):
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    p = I.square16_hubbard()
    with vmc.Context(p, 4 * nsm, seed=1, precision=vmc.MIXED, max_samples=1) as ctx:
        grid, per_sm, smem = ctx.sweep_launch()
    N = p.N
    assert smem >= 2 * 4 * N * (N + 1)          # hi and lo words of M^-1
    assert per_sm >= 2, (per_sm, smem)
    assert grid == nsm * per_sm


def test_sweep_launch_without_projection_and_with(vmc):
    import numpy as np
    from oracle.projection import momentum_weights, translations
    p = I.make_problem("c6", I.chain(6, -1), 4, U=3.0, f_full=True, jastrow="chain",
                       f_init="none", noise=0.6, seed=9, p_exchange=0.5)
    ops = momentum_weights(translations(p.lat), (0.0, 0.0))
    perm = np.array([op.perm for op, _ in ops], np.int32).reshape(len(ops), p.Ns)
    sign = np.array([op.sign for op, _ in ops]).astype(np.int8).reshape(len(ops), p.Ns)
    w = np.array([float(complex(x).real) for _, x in ops])
    with vmc.Context(p, 8, seed=1) as ctx:
        g0, o0, b0 = ctx.sweep_launch()
        assert g0 == 8 and o0 >= 1 and b0 > 0
        ctx.set_projection(perm, sign, w)
        g1, o1, b1 = ctx.sweep_launch()
        assert g1 == 8 and o1 >= 1 and b1 > 0 and b1 != b0
