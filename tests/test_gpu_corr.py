"""GPU parity of the pair-correlation measurement (vmc_measure_corr; the
physical-quantity mode of Sec. 2.2.3, estimator Eq. MC) against
oracle.physics on identical walker configurations.

Tolerances:
* plain FP64 form: every entry of the six [Ns, Ns] matrices within 1e-10 of
  max(1, |oracle|);
* mixed form (FP32 M^-1 and ratios, FP64 means): within 1e-4, the energy
  accuracy the mixed form is held to (1e-4 t per site), since E_loc is a
  sum of these entries weighted by O(1) couplings;
* diagonal kinds (n_i n_j, S^z_i S^z_j): exact (integer occupation counts);
* set configurations have cond(X) < 1e3 (FP32 ratio errors stay near
  N eps_32 cond, below the mixed tolerance); sampled ones are as drawn;
* local-energy identity (mean E_loc of the sampler = couplings x
  correlations): 1e-9 relative in FP64, 1e-4 t per site in the mixed form.
"""
import numpy as np
import pytest

from oracle import fock
from oracle.physics import local_correlation, mean_correlations
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I

from test_gpu_parity import small_problems, with_correlations

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1711_11418_gb300 import build, vmc as V
    build.build()
    return V


def corr_problems():
    d = small_problems()
    d.pop("square8")
    d["chain6_t2"] = I.make_problem("c6t2", I.chain(6, -1), 6, t2=0.4, U=3.0, f_full=True,
                                    jastrow="chain", noise=0.3, seed=2)
    d["sq4_doublons"] = I.make_problem("sq4", I.square(4, 4, 1, -1), 10, U=4.0, sub=(2, 2),
                                       jastrow="distance", f_init="none", noise=0.5, seed=5)
    return d


def conditioned_configs(p, W, seed, limit=1e3, tries=2000):
    wf = Wavefunction(p)
    out = []
    for s in range(seed, seed + tries):
        c = I.initial_configs(p.Ns, p.Ne, 1, p.local_spin, s)[0]
        X, _ = wf.X(fock.from_labels(c, p.Ns))
        if np.linalg.cond(X) < limit:
            out.append(c)
            if len(out) == W:
                return np.array(out, np.int32)
    raise RuntimeError("no well-conditioned configurations")


def occupation_means(cfg, Ns):
    """Exact n_i n_j and S^z_i S^z_j means of labelled configurations."""
    N = cfg.shape[1] // 2
    up = np.zeros((len(cfg), Ns))
    dn = np.zeros((len(cfg), Ns))
    for w, e in enumerate(cfg):
        up[w, e[:N]] = 1
        dn[w, e[N:]] = 1
    n = up + dn
    sz = 0.5 * (up - dn)
    return n.T @ n / len(cfg), sz.T @ sz / len(cfg)


def energy_from_corr(p, c):
    e = 0.0
    for i, j, t in zip(p.hop_i, p.hop_j, p.hop_t):
        e += -t * (c[0, i, j] + c[1, i, j])
    D = 0.5 * (np.diagonal(c[2]) - np.diagonal(c[0]) - np.diagonal(c[1]))
    e += float(np.asarray(p.U) @ D)
    for i, j, v in zip(p.V_i, p.V_j, p.V_val):
        e += v * c[2, i, j]
    for i, j, J in zip(p.ex_i, p.ex_j, p.ex_J):
        e += J * c[5, i, j]
    return e


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["ring8", "ring6_apbc", "heis4", "j1j2_4", "chain6_t2",
                                  "sq4_doublons"])
def test_corr_matches_oracle_small(vmc, name, form):
    p = with_correlations(corr_problems()[name], seed=1)
    W = 8
    cfg = conditioned_configs(p, W, 300)
    prec = vmc.FP64 if form == "fp64" else vmc.MIXED
    with vmc.Context(p, W, seed=5, precision=prec) as ctx:
        ctx.set_configs(cfg)
        c, ms = ctx.measure_corr(timing=True)
        ele, _ = ctx.get_configs()
    assert np.array_equal(ele, cfg)
    assert ms[0] > 0.0 and ms[1] >= ms[0]
    ref = mean_correlations(Wavefunction(p), [fock.from_labels(e, p.Ns) for e in cfg])
    tol = 1e-10 if form == "fp64" else 1e-4
    for kind in range(6):
        err = np.abs(c[kind] - ref[kind]) / np.maximum(1.0, np.abs(ref[kind]))
        assert err.max() <= tol, (kind, err.max())
    nn, szsz = occupation_means(cfg, p.Ns)
    np.testing.assert_allclose(c[2], nn, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c[3], szsz, rtol=0, atol=1e-15)


def test_corr_after_sampling_and_in_a_batch(vmc):
    """Walkers moved by the sampler (inverses updated in the sweep), and
    system 1 of a two-system batch (uneven sizes)."""
    a = with_correlations(I.ring8_hubbard(), seed=2)
    b = with_correlations(corr_problems()["sq4_doublons"], seed=3)
    W = 6
    with vmc.Context([a, b], W, seed=11) as ctx:
        ctx.sample(4, 1, 1)
        c1 = ctx.measure_corr(system=1)
        c0 = ctx.measure_corr(system=0)
        e1, _ = ctx.get_configs(system=1)
        e0, _ = ctx.get_configs(system=0)
    for p, c, ele in ((a, c0, e0), (b, c1, e1)):
        ref = mean_correlations(Wavefunction(p), [fock.from_labels(e, p.Ns) for e in ele])
        err = np.abs(c - ref) / np.maximum(1.0, np.abs(ref))
        assert err.max() <= 1e-9, err.max()


def test_corr_rejects_mlp_context(vmc):
    p = I.make_problem("r6m", I.chain(6, -1), 6, U=4.0, sub=(2, 1), jastrow="chain",
                       noise=0.2, seed=4, mlp_hidden=4)
    with vmc.Context(p, 2, seed=1) as ctx:
        with pytest.raises(vmc.VmcError) as e:
            ctx.measure_corr()
        assert e.value.code == -1
        # a system index the context does not have, at the C boundary
        buf = np.zeros(6 * p.Ns * p.Ns)
        assert ctx._L.vmc_measure_corr(ctx._h, 1, vmc._p(buf, vmc._F64P), None) == -1


def _sampled_entries(cfg_pair, Ns, rng):
    """Entries (kind, i, j) to check: for each kind, pairs where the
    estimator is non-zero on one of the two configurations, a diagonal
    entry and random pairs."""
    out = []
    N = cfg_pair.shape[1] // 2
    for e in cfg_pair:
        up = np.zeros(Ns, bool)
        dn = np.zeros(Ns, bool)
        up[e[:N]] = True
        dn[e[N:]] = True
        hop_up = [(i, j) for i in np.flatnonzero(~up) for j in np.flatnonzero(up)]
        hop_dn = [(i, j) for i in np.flatnonzero(~dn) for j in np.flatnonzero(dn)]
        swap = [(i, j) for i in np.flatnonzero(dn & ~up) for j in np.flatnonzero(up & ~dn)]
        for kind, pool in ((0, hop_up), (1, hop_dn), (4, swap), (5, swap)):
            for k in rng.choice(len(pool), 2, replace=False):
                i, j = pool[k]
                out.append((kind, int(i), int(j)))
        i, j = pool[rng.integers(len(pool))]
        out.append((5, int(j), int(i)))          # S^-_i S^+_j side of kind 5
    for kind in range(6):
        out.append((kind, int(rng.integers(Ns)), int(rng.integers(Ns))))
        d = int(rng.integers(Ns))
        out.append((kind, d, d))
    return out


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_corr_fullsize_launch_shape_two_configurations(vmc, form):
    """16x16 Hubbard (Ne = 224), 4096 walkers, the benchmark's launch shape:
    the walkers alternate between two configurations A and B, so every
    walker mean is (A + B) / 2; sampled entries of every kind against the
    oracle, the diagonal kinds in full, and the per-spin particle number."""
    p = with_correlations(I.square16_hubbard(), seed=4)
    W = 4096
    pair = conditioned_configs(p, 2, 500)
    cfg = np.array([pair[w % 2] for w in range(W)], np.int32)
    prec = vmc.FP64 if form == "fp64" else vmc.MIXED
    with vmc.Context(p, W, seed=3, precision=prec) as ctx:
        ctx.set_configs(cfg)
        c = ctx.measure_corr()
    wf = Wavefunction(p)
    ns = [fock.from_labels(e, p.Ns) for e in pair]
    rng = np.random.default_rng(7)
    tol = 1e-10 if form == "fp64" else 1e-4
    for kind, i, j in _sampled_entries(pair, p.Ns, rng):
        ref = 0.5 * (local_correlation(wf, ns[0], kind, i, j) +
                     local_correlation(wf, ns[1], kind, i, j))
        assert abs(c[kind, i, j] - ref) <= tol * max(1.0, abs(ref)), (kind, i, j, c[kind, i, j], ref)
    nn, szsz = occupation_means(pair, p.Ns)
    np.testing.assert_allclose(c[2], nn, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c[3], szsz, rtol=0, atol=1e-15)
    assert np.trace(c[0]) == pytest.approx(p.Ne // 2, abs=1e-12)
    assert np.trace(c[1]) == pytest.approx(p.Ne // 2, abs=1e-12)


@pytest.mark.parametrize("case", ["hubbard16_mixed", "hubbard16_fp64", "j1j2_16_mixed"])
def test_corr_energy_identity_fullsize(vmc, case):
    """E_loc is linear in the operators of H: the sampler's mean E_loc over
    the walkers' current configurations (the last measurement of a call is
    taken on the stored configuration) equals the couplings of H contracted
    with the measured correlations (two independent GPU code paths; at the
    16x16 sizes of the benchmark)."""
    if case.startswith("hubbard16"):
        p = I.square16_hubbard()
        W = 4096
    else:
        p = I.j1j2_heisenberg(16)
        W = 1024
    prec = vmc.FP64 if case.endswith("fp64") else vmc.MIXED
    with vmc.Context(p, W, seed=21, precision=prec, max_samples=1) as ctx:
        ctx.sample(3, 1, 1)
        E, _ = ctx.get_samples()
        c = ctx.measure_corr()
    e_corr = energy_from_corr(p, c)
    if prec == vmc.FP64:
        assert e_corr == pytest.approx(E.mean(), rel=1e-9)
    else:
        assert abs(e_corr - E.mean()) <= 1e-4 * p.Ns
