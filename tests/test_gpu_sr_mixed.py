"""GPU checks of the mixed-precision SR solve (iterative refinement in FP64
with an FP32 inverse of the Jacobi-scaled S~ as the correction operator,
FP64 Cholesky fallback).

Pins: on the oracle's SR problem the update equals the oracle's Cholesky
solution (Sec. 3.3.2) within 1e-9; at the 16x16 workload size the
refined solution's FP64 backward error |g - S~ x| / |g| is below 1e-11 with
S~ taken from the library itself; an ill-conditioned S~ (cond ~ 1e10, beyond
FP32) triggers the fallback, whose result is the FP64 Cholesky's.
"""
import numpy as np
import pytest

from oracle.sr import sr_step
from paper_1711_11418_gb300 import inputs as I

from test_gpu_parity import rel_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


def test_mixed_ir_matches_oracle_cholesky(vmc):
    p = I.ring8_hubbard()
    E, O = I.random_samples(1000, p.Np, seed=11)
    with vmc.Context(p, 10, seed=1, max_samples=100) as ctx:
        ctx.set_samples(E, O)
        p0 = ctx.get_params()
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-13)
        d_gpu = ctx.get_params() - p0
    d_ref, _ = sr_step(E, O, 0.05, 1e-3, 0.0, "cholesky")
    assert rep["fallback"] == 0
    assert 1 <= rep["cg_iters"] <= 16
    assert rep["rel_residual"] <= 1e-13
    assert rel_close(d_gpu, d_ref, rtol=1e-9)


@pytest.mark.parametrize("rows,Np", [(2049, 300), (4096, 1069)])
def test_mixed_ir_backward_error_workload_size(vmc, rows, Np):
    """Mixed context (split-BF16 tensor-core S), SR dimensions up to the
    16x16 Hubbard workload's: |g - S~ x| / |g| < 1e-11 in FP64 with S~ and g
    from the library, and the update agrees with the FP64 Cholesky's."""
    p = I.square16_hubbard() if Np == 1069 else I.make_problem(
        "sq", I.square(10, 10, 1, -1), 88, U=4.0, sub=(2, 2), jastrow="distance", noise=0.05,
        seed=2)
    Np = p.Np
    W = 16
    S_per = (rows + W - 1) // W
    E, O = I.random_samples(W * S_per, Np, seed=5)
    with vmc.Context(p, W, seed=1, precision=vmc.MIXED, max_samples=S_per) as ctx:
        ctx.set_samples(E, O)
        St, g = ctx.get_sr_matrices(1e-3, 0.0)
        p0 = ctx.get_params()
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-12)
        x = -(ctx.get_params() - p0) / 0.05
        ctx.set_params(p0)
        ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.CHOLESKY)
        x_chol = -(ctx.get_params() - p0) / 0.05
    assert rep["fallback"] == 0
    res = np.linalg.norm(g - St @ x) / np.linalg.norm(g)
    assert res < 1e-11, res
    assert rel_close(x, x_chol, rtol=1e-7)


def test_mixed_ir_falls_back_when_fp32_cannot(vmc):
    """Nearly collinear columns, no shift: cond(S~) ~ 1e10, the FP32 inverse
    is useless, the refinement does not converge and the FP64 Cholesky
    solves instead (the result of asking for it, up to the atomic-order
    rounding of the S build amplified by cond(S~))."""
    p = I.ring8_hubbard()
    rng = np.random.default_rng(3)
    E, O = I.random_samples(1000, p.Np, seed=12)
    O = O.copy()
    O[:, 1] = O[:, 0] + 1e-5 * rng.standard_normal(O.shape[0])
    with vmc.Context(p, 10, seed=1, max_samples=100) as ctx:
        ctx.set_samples(E, O)
        p0 = ctx.get_params()
        rep = ctx.sr_step(0.05, 0.0, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-12)
        d_ir = ctx.get_params() - p0
        ctx.set_params(p0)
        ctx.sr_step(0.05, 0.0, 0.0, solver=vmc.CHOLESKY)
        d_ch = ctx.get_params() - p0
    assert rep["fallback"] == 1
    assert rel_close(d_ir, d_ch, rtol=1e-4)


def test_mixed_ir_on_sampled_overlap_matrix(vmc):
    """S~ from the mixed form's own samples of the 8x8 Hubbard model (shift
    1e-3, as in the benchmark): the refined solution's FP64 backward error is
    below 1e-11, or the FP64 Cholesky took over."""
    p = I.square8_hubbard()
    W, S = 256, 8
    with vmc.Context(p, W, seed=3, precision=vmc.MIXED, max_samples=S) as ctx:
        ctx.sample(5, S, 1)
        St, g = ctx.get_sr_matrices(1e-3, 0.0)
        p0 = ctx.get_params()
        rep = ctx.sr_step(0.05, 1e-3, 0.0, solver=vmc.MIXED_IR, cg_eps=1e-12)
        x = -(ctx.get_params() - p0) / 0.05
    res = np.linalg.norm(g - St @ x) / np.linalg.norm(g)
    assert res < (1e-11 if rep["fallback"] == 0 else 1e-8), (res, rep)


def test_mixed_form_srcg_matches_oracle(vmc):
    """Mixed form, CG with the SR-CG product (S never formed), whose two
    passes over the FP32 samples sum FP32 products in FP32 over 16 terms and
    in FP64 beyond: the update equals the oracle's Cholesky solution of the
    same (FP32-rounded) samples within 1e-5, for 300 parameters and 2049
    rows (ragged against the 16-term chunks)."""
    base = I.ring8_hubbard()
    Np = 300
    n_f = Np - base.n_g - base.n_v
    p = base.copy_with(n_f=n_f, f_idx=np.arange(64, dtype=np.int32), f_sign=np.ones(64, np.int8),
                       params=np.concatenate([base.params[:3],
                                              np.random.default_rng(0).uniform(-1, 1, n_f)]))
    rows, W = 2049, 16
    E, O = I.random_samples(rows, Np, seed=31)
    O[:, : Np // 3] += 0.5
    with vmc.Context(p, W, seed=1, precision=vmc.MIXED, max_samples=(rows + W - 1) // W) as ctx:
        ctx.set_samples(E, O)
        p0 = ctx.get_params()
        rep = ctx.sr_step(0.05, 1e-3, 1e-4, solver=vmc.CG, cg_eps=1e-9, cg_kmax=1000)
        d_gpu = ctx.get_params() - p0
    d_ref, _ = sr_step(E, O.astype(np.float32).astype(np.float64), 0.05, 1e-3, 1e-4, "cholesky")
    assert rep["cg_iters"] > 0
    assert rel_close(d_gpu, d_ref, rtol=1e-5)
