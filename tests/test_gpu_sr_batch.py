"""vmc_sr_step_all: one SR step for every system of a batch, the work of all
systems enqueued before the host waits.  Pin: the parameter updates and
reports equal those of vmc_sr_step called system by system on an identical
context (same kernels in the same order per system), for the mixed form with
the refinement solve and the FP64 form with the Cholesky solve."""
import numpy as np
import pytest

from paper_1711_11418_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


W, S = 16, 16


def stepped(vmc, probs, precision, solver, batched):
    """Identical seeded samples in every system (sampled O_k rows differ at the
    rounding level between runs: shared-memory atomic sums), one SR step."""
    with vmc.Context(probs, W, seed=13, precision=precision, max_samples=S) as ctx:
        for s, p in enumerate(probs):
            E, O = I.random_samples(W * S, p.Np, seed=100 + s)
            O[:, : p.Np // 3] += 0.3
            ctx.set_samples(E, O, system=s)
        p0 = [ctx.get_params(s) for s in range(len(probs))]
        if batched:
            reps = ctx.sr_step_all(0.05, 1e-3, 1e-4, solver=solver, cg_eps=1e-12)
        else:
            reps = [ctx.sr_step(0.05, 1e-3, 1e-4, solver=solver, cg_eps=1e-12, system=s)
                    for s in range(len(probs))]
        d = [ctx.get_params(s) - p0[s] for s in range(len(probs))]
        ctx.sample(0, 1, 1)   # the next sampling rebuilds every system's inverses
        e = [ctx.measure(s)["energy"] for s in range(len(probs))]
    return d, reps, e


@pytest.mark.parametrize("prec,solver", [("MIXED", "MIXED_IR"), ("FP64", "CHOLESKY")])
def test_sr_step_all_equals_per_system_steps(vmc, prec, solver):
    probs = I.batched_hubbard(8, seed=2)
    precision, solv = getattr(vmc, prec), getattr(vmc, solver)
    d1, r1, e1 = stepped(vmc, probs, precision, solv, False)
    d2, r2, e2 = stepped(vmc, probs, precision, solv, True)
    for s in range(len(probs)):
        assert np.allclose(d2[s], d1[s], rtol=1e-12, atol=1e-15), s
        assert r2[s]["energy"] == pytest.approx(r1[s]["energy"], rel=1e-13)
        assert r2[s]["norm_g"] == pytest.approx(r1[s]["norm_g"], rel=1e-12)
        assert r2[s]["cg_iters"] == r1[s]["cg_iters"]
        assert r2[s]["fallback"] == r1[s]["fallback"]
        assert r2[s]["n_params"] == probs[s].Np
        assert np.isfinite(e2[s])


def test_sr_step_all_cg_and_state(vmc):
    probs = I.batched_hubbard(4, seed=3)
    with vmc.Context(probs, 4, seed=1, precision=vmc.MIXED, max_samples=2) as ctx:
        with pytest.raises(vmc.VmcError):
            ctx.sr_step_all(0.05, 1e-3, 1e-4, solver=vmc.MIXED_IR)   # no samples yet
        ctx.sample(2, 2, 1)
        reps = ctx.sr_step_all(0.05, 1e-3, 1e-4, solver=vmc.CG, cg_eps=1e-8, cg_kmax=200)
        assert len(reps) == len(probs)
        assert all(r["cg_iters"] > 0 for r in reps)
