"""GPU quantum-number projection (vmc_set_projection; Sec. 3.2.2, Eqs. momP and
pointP; boundary signs of App. A) against the oracle's ProjectedWavefunction
on identical seeded inputs, FP64 form: projected Pfaffian ratios within
1e-10, Markov chains bit-exact with E_loc and O_k rows within 1e-10, the SR
step from the GPU's samples equal to the oracle's; the mixed form within 1e-4
per site.  The operations are the translations (anti-periodic signs
included) with real characters K = 0 and K = pi, and on the anti-periodic
3x3 lattice the translations composed with the point group: the same cases
the oracle's own pins cover on the CPU (tests/test_oracle_projection.py).
"""
import math

import numpy as np
import pytest

from oracle import fock
from oracle.projection import ProjectedWavefunction, combine, momentum_weights, point_ops, translations
from oracle.sampler import run_sampling
from oracle.sr import sr_step
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I

from helpers import condition_ok, oracle_ratio, random_moves

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


def chain6():
    p = I.make_problem("c6", I.chain(6, -1), 4, U=3.0, f_full=True, jastrow="chain",
                       f_init="none", noise=0.6, seed=9, p_exchange=0.5)
    p.params[:3] = [-0.4, 0.2, -0.1]
    return p


def square3():
    p = I.make_problem("s3", I.square(3, 3, -1, -1), 4, U=2.0, sub=(1, 1), f_full=True,
                       f_init="none", noise=0.5, seed=2, p_exchange=0.5)
    p.params[0] = -0.3
    return p


def heis4():
    return I.make_problem("h4", I.chain(4, 1), 4, t=0.0, J1=1.0, local_spin=True, f_full=True,
                          gutzwiller=False, noise=0.3, seed=6)


def ops_arrays(ops, Ns):
    perm = np.array([op.perm for op, _ in ops], np.int32).reshape(len(ops), Ns)
    sign = np.array([op.sign for op, _ in ops]).astype(np.int8).reshape(len(ops), Ns)
    w = np.array([float(complex(w).real) for _, w in ops])
    return perm, sign, w


def cases():
    c6 = chain6()
    tr6 = translations(c6.lat)
    s3 = square3()
    pts = point_ops(s3.lat)
    h4 = heis4()
    return {
        "chain6_K0": (c6, momentum_weights(tr6, (0.0, 0.0))),
        "chain6_Kpi": (c6, momentum_weights(tr6, (math.pi, 0.0))),
        "square3_K0_A1": (s3, combine(momentum_weights(translations(s3.lat), (0.0, 0.0)),
                                      [(op, 1.0 / len(pts)) for op, _ in pts])),
        "heis4_K0": (h4, momentum_weights(translations(h4.lat), (0.0, 0.0))),
    }


def projected(p, ops):
    ops = [(op, float(complex(w).real)) for op, w in ops]
    return ProjectedWavefunction(Wavefunction(p), ops), ops


def good_configs(p, pw, W, seed):
    base = Wavefunction(p)
    out, s = [], seed
    while len(out) < W:
        c = I.initial_configs(p.Ns, p.Ne, 1, p.local_spin, s)[0]
        s += 1
        n = fock.from_labels(c, p.Ns)
        if condition_ok(base, c) and abs(pw.amplitude(n)) > 1e-8 * math.exp(
                base.amplitude_slog(n)[1]):
            out.append(c)
    return np.array(out, np.int32)


@pytest.mark.parametrize("name", sorted(cases()))
def test_projected_ratios(vmc, name):
    p, ops = cases()[name]
    pw, ops = projected(p, ops)
    cfg = good_configs(p, pw, 2, 30)
    rng = np.random.default_rng(5)
    with vmc.Context(p, 2, seed=3) as ctx:
        ctx.set_projection(*ops_arrays(ops, p.Ns))
        ctx.set_configs(cfg)
        for w in range(2):
            moves = random_moves(rng, cfg[w], p.N, p.Ns, p.local_spin, 16)
            got = ctx.eval_ratios(w, moves)
            ref = np.array([oracle_ratio(pw, cfg[w], m) for m in moves])
            big = np.abs(ref) > 1e-8
            assert big.sum() >= 4
            assert np.all(np.abs(got[big] - ref[big]) <= RTOL * np.abs(ref[big]) + 1e-13), (
                got[big], ref[big])


@pytest.mark.parametrize("name", sorted(cases()))
def test_projected_chains_energies_and_log_derivatives(vmc, name):
    p, ops = cases()[name]
    pw, ops = projected(p, ops)
    W, S = 3, 3
    cfg = good_configs(p, pw, W, 50)
    with vmc.Context(p, W, seed=21, max_samples=S) as ctx:
        ctx.set_projection(*ops_arrays(ops, p.Ns))
        ctx.set_configs(cfg)
        ctx.sample(1, S, 1)
        ele, ctr = ctx.get_configs()
        E, O = ctx.get_samples()
        p0 = ctx.get_params()
        ctx.sr_step(0.05, 1e-3, 1e-4, solver=vmc.CHOLESKY)
        d = ctx.get_params() - p0
    ref = run_sampling(pw, cfg, 21, 0, 1, S, 1, p.p_exchange)
    assert np.array_equal(ele, ref["ele"])
    assert np.array_equal(ctr, ref["counters"])
    assert np.max(np.abs(E - ref["E"])) <= RTOL * max(1.0, np.max(np.abs(ref["E"])))
    assert np.max(np.abs(O - ref["O"])) <= RTOL * max(1.0, np.max(np.abs(ref["O"])))
    dref, _ = sr_step(ref["E"], ref["O"], 0.05, 1e-3, 1e-4, "cholesky")
    assert np.max(np.abs(d - dref)) <= 1e-8 * max(1e-12, np.max(np.abs(dref)))


def test_projected_mixed_form_close_to_fp64(vmc):
    p, ops = cases()["square3_K0_A1"]
    pw, ops = projected(p, ops)
    W = 4
    cfg = good_configs(p, pw, W, 70)
    res = {}
    for prec in (vmc.FP64, vmc.MIXED):
        with vmc.Context(p, W, seed=2, precision=prec, max_samples=1) as ctx:
            ctx.set_projection(*ops_arrays(ops, p.Ns))
            ctx.set_configs(cfg)
            ctx.sample(0, 1, 0)
            res[prec] = ctx.get_samples()
    assert np.max(np.abs(res[vmc.FP64][0] - res[vmc.MIXED][0])) / p.Ns < 1e-4


def test_projection_rejections(vmc):
    p, ops = cases()["chain6_K0"]
    perm, sign, w = ops_arrays([(op, float(complex(x).real)) for op, x in ops], p.Ns)
    with vmc.Context(p, 2, seed=1) as ctx:
        bad = perm.copy()
        bad[1, 0] = bad[1, 1]                      # not a permutation
        with pytest.raises(vmc.VmcError):
            ctx.set_projection(bad, sign, w)
        ctx.set_projection(perm, sign, w)
        with pytest.raises(vmc.VmcError):
            ctx.measure_corr()
        with pytest.raises(vmc.VmcError):
            ctx.set_delay(4)
        ctx.set_projection(np.zeros((0, p.Ns)), np.zeros((0, p.Ns)), np.zeros(0))
        ctx.measure_corr()                         # unprojected again


@pytest.mark.parametrize("precision,rtol", [("MIXED", 1e-5), ("FP64", 1e-10)])
def test_identity_projection_equals_plain_state_full_size(vmc, precision, rtol):
    """Projection onto the identity alone (N_g = 1, weight 1) is the plain
    state.  On the 16x16 lattice with next-nearest hops (about 1000 hop
    terms with a move per configuration: two chunks of the mixed form's
    term listing) the projected measurement's E_loc and O_k equal the plain
    measurement's on the same configurations."""
    prec = getattr(vmc, precision)
    p = I.make_problem("s16t2", I.square(16, 16, -1, -1), 224, U=8.0, t2=-0.3, sub=(2, 2),
                       jastrow="distance", f_init="none", noise=0.5, seed=3)
    p.params[:p.n_g + p.n_v] = np.random.default_rng(4).uniform(-0.3, 0.1, p.n_g + p.n_v)
    W = 32
    cfg = I.initial_configs(p.Ns, p.Ne, W, False, 77)
    res = []
    for proj in (False, True):
        with vmc.Context(p, W, seed=5, precision=prec, max_samples=1) as ctx:
            if proj:
                ctx.set_projection(np.arange(p.Ns, dtype=np.int32)[None, :],
                                   np.ones((1, p.Ns), np.int8), np.ones(1))
            ctx.set_configs(cfg)
            ctx.sample(0, 1, 0)
            res.append(ctx.get_samples())
    (E0, O0), (E1, O1) = res
    assert np.allclose(E1, E0, rtol=rtol, atol=rtol * np.max(np.abs(E0)))
    assert np.allclose(O1, O0, rtol=rtol, atol=rtol * max(1.0, np.max(np.abs(O0))))
