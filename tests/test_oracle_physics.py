"""Pins of the physical-quantity oracle (oracle.physics) against what the
mathematics fixes: Wick's theorem for the U = 0 Slater state, the two-site
singlet and triplet, the total-spin sum rule of a singlet wave function, the
local-energy identity (Eq. MC applied to H term by term), and particle-number
sum rules.  No GPU.
"""
import numpy as np
import pytest

from oracle import fock
from oracle.hamiltonian import local_energy
from oracle.physics import (doublon_density, exact_correlations, local_correlation,
                            local_correlations, mean_correlations, nn_spin_correlation,
                            structure_factor)
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I


def _hopping_matrix(p):
    h = np.zeros((p.Ns, p.Ns))
    for i, j, t in zip(p.hop_i, p.hop_j, p.hop_t):
        h[i, j] += -t
    return h


def test_free_fermion_correlations_follow_wick():
    """U = 0, no correlation factors, f from the lowest orbitals of the
    hopping matrix (closed shell): psi is a product of two Slater
    determinants, so every correlation is a closed form in the one-body
    density matrix rho = Phi Phi^T (Wick's theorem)."""
    p = I.make_problem("ff6", I.chain(6, -1), 4, U=0.0, f_full=True, gutzwiller=False,
                       noise=0.0)
    h = _hopping_matrix(p)
    w, V = np.linalg.eigh(h)
    N = p.Ne // 2
    assert w[N] - w[N - 1] > 0.5          # closed shell: rho is unique
    rho = V[:, :N] @ V[:, :N].T
    d = np.diag(rho)
    eye = np.eye(p.Ns)
    c = exact_correlations(Wavefunction(p))
    np.testing.assert_allclose(c[0], rho, atol=1e-12)
    np.testing.assert_allclose(c[1], rho, atol=1e-12)
    nn = 4 * np.outer(d, d) - 2 * rho ** 2 + 2 * eye * d
    np.testing.assert_allclose(c[2], nn, atol=1e-12)
    szsz = 0.5 * (eye * d - rho ** 2)
    np.testing.assert_allclose(c[3], szsz, atol=1e-12)
    spsm = np.where(eye > 0, d * (1 - d), -rho ** 2)
    np.testing.assert_allclose(c[4], spsm, atol=1e-12)
    np.testing.assert_allclose(c[5], szsz + spsm, atol=1e-12)
    # D = (1/Ns) sum_i rho_ii^2 (up and down sectors independent)
    assert doublon_density(c) == pytest.approx(float(np.sum(d * d)) / p.Ns, abs=1e-12)


def _two_site(f01, f10):
    p = I.make_problem("s2", I.chain(4, 1), 2, t=0.0, J1=1.0, local_spin=True,
                       gutzwiller=False, f_full=True, noise=0.0, f_init="none")
    return p.copy_with(lat=I.Lattice(2, 1), ex_i=np.array([0], np.int32),
                       ex_j=np.array([1], np.int32), ex_J=np.array([1.0]), U=np.zeros(2),
                       f_idx=np.array([-1, 0, 1, -1], np.int32), f_sign=np.ones(4, np.int8),
                       n_f=2, params=np.array([f01, f10]), g_idx=np.full(2, -1, np.int32),
                       n_g=0, v_idx=np.full(4, -1, np.int32), n_v=0)


@pytest.mark.parametrize("f10,ss,spsm", [(0.7, -0.75, -0.5), (-0.7, 0.25, 0.5)])
def test_two_site_singlet_and_triplet(f10, ss, spsm):
    """Symmetric f on two sites is the singlet, antisymmetric f the m = 0
    triplet: <S_0.S_1> = -3/4 or +1/4 on both configurations (an eigenstate
    has a constant local estimator), <S^+_0 S^-_1> = -1/2 or +1/2."""
    wf = Wavefunction(_two_site(0.7, f10))
    for ele in ([0, 1], [1, 0]):
        loc = local_correlations(wf, fock.from_labels(ele, 2))
        assert loc[5, 0, 1] == pytest.approx(ss, abs=1e-14)
        assert loc[5, 1, 0] == pytest.approx(ss, abs=1e-14)
        assert loc[3, 0, 1] == pytest.approx(-0.25, abs=1e-14)
    c = exact_correlations(wf)
    assert c[4, 0, 1] == pytest.approx(spsm, abs=1e-14)
    assert c[4, 1, 0] == pytest.approx(spsm, abs=1e-14)
    assert c[5, 0, 0] == pytest.approx(0.75, abs=1e-14)


def _correlated_chain(symmetric, seed=3):
    """6-site Hubbard chain at half filling with random Gutzwiller, Jastrow
    and f (no local-spin constraint)."""
    p = I.make_problem("c6", I.chain(6, -1), 6, U=4.0, f_full=True, jastrow="chain",
                       f_init="none", noise=0.0)
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1, 1, (6, 6))
    if symmetric:
        f = 0.5 * (f + f.T)
    params = np.concatenate([[-0.6], [0.3, -0.2], f.reshape(-1)])
    return p.copy_with(params=params)


def test_singlet_sum_rule():
    """Symmetric f makes the pair product a total singlet and the Gutzwiller
    and Jastrow factors depend on charge only, so psi is a singlet:
    sum_ij <S_i.S_j> = S(S+1) = 0 and sum_ij <S^+_i S^-_j> = 0.  A random
    non-symmetric f mixes in triplets and the sums are positive."""
    c = exact_correlations(Wavefunction(_correlated_chain(True)))
    assert abs(c[5].sum()) < 1e-12
    assert abs(c[4].sum()) < 1e-12
    assert abs(c[3].sum()) < 1e-12          # S^z_tot = 0 on every configuration
    c2 = exact_correlations(Wavefunction(_correlated_chain(False)))
    assert c2[5].sum() > 1e-2
    assert c2[4].sum() > 1e-2


def _energy_from_correlations(p, loc):
    e = 0.0
    for i, j, t in zip(p.hop_i, p.hop_j, p.hop_t):
        e += -t * (loc[0, i, j] + loc[1, i, j])
    D = 0.5 * (np.diagonal(loc[2]) - np.diagonal(loc[0]) - np.diagonal(loc[1]))
    e += float(np.asarray(p.U) @ D)
    for i, j, v in zip(p.V_i, p.V_j, p.V_val):
        e += v * loc[2, i, j]
    for i, j, J in zip(p.ex_i, p.ex_j, p.ex_J):
        e += J * loc[5, i, j]
    return e


@pytest.mark.parametrize("which", ["ring8_V", "heis4x4", "chain6_t2"])
def test_local_energy_identity(which):
    """E_loc(x) is linear in the operators of H, so on every configuration it
    equals the sum of the local correlations weighted by H's couplings (the
    energy estimator is pinned against exact diagonalisation elsewhere)."""
    if which == "ring8_V":
        p = I.ring8_hubbard()
        p = p.copy_with(V_i=np.arange(8, dtype=np.int32),
                        V_j=((np.arange(8) + 1) % 8).astype(np.int32), V_val=np.full(8, 0.7))
        p.params[:3] = [-0.5, 0.2, -0.1]
    elif which == "heis4x4":
        p = I.heisenberg_square(4)
    else:
        p = I.make_problem("c6t2", I.chain(6, -1), 6, t2=0.4, U=3.0, f_full=True,
                           jastrow="chain", noise=0.3, seed=2)
    wf = Wavefunction(p)
    cfgs = I.initial_configs(p.Ns, p.Ne, 3, p.local_spin, 17)
    for ele in cfgs:
        n = fock.from_labels(ele, p.Ns)
        loc = local_correlations(wf, n)
        e = local_energy(wf, n)
        assert _energy_from_correlations(p, loc) == pytest.approx(e, rel=1e-11, abs=1e-11)


def test_local_estimators_act_on_the_ket_and_conserve_particles():
    """Eq. MC applies A to |x>: c^dag_i c_j is nonzero on x only if site j
    holds the electron and site i is free (i != j); n_i n_j, S^z S^z and the
    diagonal one-body terms are the occupations."""
    p = I.ring8_hubbard()
    wf = Wavefunction(p)
    ele = I.initial_configs(p.Ns, p.Ne, 1, False, 4)[0]
    n = fock.from_labels(ele, p.Ns)
    loc = local_correlations(wf, n)
    N = p.Ne // 2
    up = np.zeros(p.Ns)
    dn = np.zeros(p.Ns)
    up[ele[:N]] = 1
    dn[ele[N:]] = 1
    for s, occ in ((0, up), (1, dn)):
        g = loc[s]
        np.testing.assert_array_equal(np.diagonal(g), occ)
        off = g - np.diag(np.diagonal(g))
        allowed = np.outer(1 - occ, occ)
        assert np.all(off[allowed == 0] == 0.0)
        assert np.count_nonzero(off) > 0
    nocc = up + dn
    np.testing.assert_array_equal(loc[2].sum(axis=1), nocc * p.Ne)
    assert abs(loc[3].sum()) < 1e-15


def test_structure_factor_sum_rules():
    """k = 0: N(0) = Ne^2 / Ns for fixed particle number, S(0) = 0 for a
    singlet; S_nn of the two-site singlet (one bond) is -3/4."""
    p = _correlated_chain(True)
    c = exact_correlations(Wavefunction(p))
    R = np.arange(p.Ns, dtype=np.float64)[:, None]
    assert structure_factor(c[2], R, [0.0]) == pytest.approx(p.Ne ** 2 / p.Ns, abs=1e-12)
    assert abs(structure_factor(c[5], R, [0.0])) < 1e-12
    ks = 2 * np.pi * np.arange(p.Ns) / p.Ns
    # sum over the Brillouin zone of S(k) = sum_i <S_i.S_i> (Parseval)
    tot = sum(structure_factor(c[5], R, [k]) for k in ks)
    assert tot == pytest.approx(float(np.trace(c[5])), abs=1e-11)
    c2 = exact_correlations(Wavefunction(_two_site(0.7, 0.7)))
    assert nn_spin_correlation(c2[5], [0], [1]) == pytest.approx(-0.75, abs=1e-14)


def test_mean_over_configurations_is_the_average_of_local_values():
    p = I.ring8_hubbard()
    wf = Wavefunction(p)
    cfgs = [fock.from_labels(e, p.Ns) for e in I.initial_configs(p.Ns, p.Ne, 3, False, 8)]
    m = mean_correlations(wf, cfgs)
    ref = sum(local_correlations(wf, n) for n in cfgs) / 3
    np.testing.assert_allclose(m, ref, rtol=0, atol=1e-15)


def test_single_entry_matches_dense():
    p = I.make_problem("c6t2", I.chain(6, -1), 6, t2=0.4, U=3.0, f_full=True, jastrow="chain",
                       noise=0.3, seed=2)
    wf = Wavefunction(p)
    n = fock.from_labels(I.initial_configs(p.Ns, p.Ne, 1, False, 3)[0], p.Ns)
    dense = local_correlations(wf, n)
    for kind in range(6):
        for i, j in ((0, 3), (2, 2), (5, 1)):
            assert local_correlation(wf, n, kind, i, j) == dense[kind, i, j]


def test_spin_swap_closed_form():
    """The identity the pair-correlation kernel uses for a spin swap (up
    electron n on site a, down electron m on site b): with B = M^-1,
    det M'/det M = G_up[b, n] G_dn[a, m] - B_mn (T[b, a] - f(b, a)), where
    G_up[b, :] = f(b, r_dn) B, G_dn[a, m] = B[m, :] f(r_up, a) and
    T[b, a] = G_up[b, :] f(r_up, a); against direct determinants."""
    rng = np.random.default_rng(0)
    Ns, N = 10, 4
    f = rng.standard_normal((Ns, Ns))
    checked = 0
    for _ in range(300):
        up = list(rng.permutation(Ns)[:N])
        dn = list(rng.permutation(Ns)[:N])
        M = f[np.ix_(up, dn)]
        if abs(np.linalg.det(M)) < 1e-6:
            continue
        B = np.linalg.inv(M)
        ns = [k for k in range(N) if up[k] not in dn]
        ms = [k for k in range(N) if dn[k] not in up]
        if not ns or not ms:
            continue
        n, m = ns[0], ms[0]
        a, b = up[n], dn[m]
        up2, dn2 = list(up), list(dn)
        up2[n], dn2[m] = b, a
        direct = np.linalg.det(f[np.ix_(up2, dn2)]) / np.linalg.det(M)
        gu = f[b, dn] @ B
        gd = B[m, :] @ f[up, a]
        T = gu @ f[up, a]
        assert gu[n] * gd - B[m, n] * (T - f[b, a]) == pytest.approx(direct, rel=1e-9, abs=1e-9)
        checked += 1
    assert checked > 100
