"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value
printed in the paper (tests/golden), a closed form, an identity, brute
force on tiny inputs, or a published known-answer vector.
"""
import math
import os

import numpy as np
import pytest

from oracle import fock
from oracle.exact import enumerate_expectations
from oracle.hamiltonian import (basis, ground_state_energy, hamiltonian_matrix,
                                hamiltonian_matrix_vec, local_energy)
from oracle.pfaffian import pfaffian, pfaffian_expand, pfaffian_slog
from oracle.philox import philox4x32_10
from oracle.sampler import run_sampling
from oracle.sr import cg, shifted, solve_cholesky, sr_matrices, sr_step, srcg_matvec
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


def skew(rng, n):
    A = rng.standard_normal((n, n))
    return A - A.T


def free_fermion_energy(Lx, Ly, bcx, bcy, N, t=1.0):
    """Textbook U = 0 energy: 2 spins x lowest N of -2t(cos kx + cos ky)."""
    kx = (2 * np.pi * np.arange(Lx) + (np.pi if bcx < 0 else 0.0)) / Lx
    if Ly == 1:
        eps = -2 * t * np.cos(kx)
    else:
        ky = (2 * np.pi * np.arange(Ly) + (np.pi if bcy < 0 else 0.0)) / Ly
        eps = (-2 * t * (np.cos(kx)[:, None] + np.cos(ky)[None, :])).ravel()
    return 2.0 * np.sort(eps)[:N].sum()


# --------------------------------------------------------------------------
# Philox (published known-answer vectors)
# --------------------------------------------------------------------------
def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox_kat.txt")):
        if line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        assert philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10])


# --------------------------------------------------------------------------
# Pfaffian (Sec. 3.2.1: Pf^2 = det; Appendix C: Pf(B A B^T) = det B Pf A)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_pfaffian_matches_definition(n):
    rng = np.random.default_rng(n)
    A = skew(rng, n)
    assert pfaffian(A) == pytest.approx(pfaffian_expand(A), rel=1e-12)


def test_pfaffian_closed_form_4x4():
    rng = np.random.default_rng(4)
    a = skew(rng, 4)
    ref = a[0, 1] * a[2, 3] - a[0, 2] * a[1, 3] + a[0, 3] * a[1, 2]
    assert pfaffian(a) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("n", [10, 20, 40])
def test_pfaffian_squared_is_det(n):
    rng = np.random.default_rng(100 + n)
    A = skew(rng, n)
    s, l = pfaffian_slog(A)
    sd, ld = np.linalg.slogdet(A)
    assert sd > 0
    assert 2 * l == pytest.approx(ld, rel=1e-11, abs=1e-10)


def test_pfaffian_congruence():
    rng = np.random.default_rng(7)
    A = skew(rng, 8)
    B = rng.standard_normal((8, 8))
    assert pfaffian(B @ A @ B.T) == pytest.approx(np.linalg.det(B) * pfaffian(A), rel=1e-10)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_pfaffian_block_identity(N):
    """Pf [[0, M], [-M^T, 0]] = (-1)^{N(N-1)/2} det M (anti-parallel form)."""
    rng = np.random.default_rng(N)
    M = rng.standard_normal((N, N))
    X = np.zeros((2 * N, 2 * N))
    X[:N, N:] = M
    X[N:, :N] = -M.T
    assert pfaffian(X) == pytest.approx((-1) ** (N * (N - 1) // 2) * np.linalg.det(M), rel=1e-11)


def test_pfaffian_zero():
    A = np.zeros((4, 4))
    A[0, 1], A[1, 0] = 1.0, -1.0
    assert pfaffian(A) == 0.0


def test_pair_state_expansion_is_pfaffian():
    """<x|[sum F_IJ c+_I c+_J]^{Ne/2}|0> = (Ne/2)! Pf(X), X_IJ = F_IJ - F_JI,
    by expanding the pair operator power in the Fock basis (Sec. 3.2.1)."""
    rng = np.random.default_rng(11)
    norb, Ne = 6, 4
    F = rng.standard_normal((norb, norb))
    state = {0: 1.0}
    for _ in range(Ne // 2):
        new = {}
        for n, a in state.items():
            for Ii in range(norb):
                for J in range(norb):
                    r = fock.apply_string([("+", Ii), ("+", J)], (a * F[Ii, J], n))
                    if r is not None:
                        new[r[1]] = new.get(r[1], 0.0) + r[0]
        state = new
    assert len(state) == math.comb(norb, Ne)
    for n, amp in state.items():
        orbs = fock.occupied(n, norb)
        Fs = F[np.ix_(orbs, orbs)]
        assert amp == pytest.approx(math.factorial(Ne // 2) * pfaffian(Fs - Fs.T), rel=1e-11)


def test_labelled_sign_matches_operator_order():
    """|x_labelled> = label_sign * |x_canonical>, built with the operators."""
    rng = np.random.default_rng(3)
    Ns, N = 5, 2
    for _ in range(10):
        ele = list(rng.choice(Ns, N, replace=False)) + list(rng.choice(Ns, N, replace=False))
        st = (1.0, 0)
        for k in reversed(range(2 * N)):
            st = fock.cdag(int(ele[k]) + (Ns if k >= N else 0), st)
        assert st[1] == fock.from_labels(ele, Ns)
        assert st[0] == fock.label_sign(ele, Ns)


# --------------------------------------------------------------------------
# Hamiltonian conventions and ED
# --------------------------------------------------------------------------
def test_heisenberg_4x4_ed_matches_paper():
    ref = golden("paper_values.txt")["heisenberg_4x4_ed_energy_per_site"]
    p = I.heisenberg_square(4)
    assert ground_state_energy(p) / 16 == pytest.approx(ref, abs=5e-9)


def test_heisenberg_ring4_closed_form():
    lat = I.chain(4, 1)
    p = I.make_problem("h4", lat, 4, t=0.0, J1=1.0, local_spin=True, sub=(1, 1),
                       gutzwiller=False)
    assert ground_state_energy(p) == pytest.approx(-2.0, abs=1e-12)


@pytest.mark.parametrize("U", [0.0, 2.0, 8.0])
def test_hubbard_two_site_closed_form(U):
    """Two-site Hubbard, two electrons: E0 = (U - sqrt(U^2 + 16 t^2)) / 2."""
    p = I.make_problem("d2", I.chain(4, 1), 2, U=U)
    p = p.copy_with(lat=I.Lattice(2, 1), hop_i=np.array([0, 1], np.int32),
                    hop_j=np.array([1, 0], np.int32), hop_t=np.array([1.0, 1.0]),
                    U=np.full(2, U))
    assert ground_state_energy(p) == pytest.approx((U - math.sqrt(U * U + 16)) / 2, abs=1e-12)


def test_vectorised_and_operator_hamiltonians_agree():
    p = I.make_problem("r6", I.chain(6, -1), 6, U=3.0, sub=(2, 1), jastrow="chain")
    st = basis(6, 3, 3)
    A = hamiltonian_matrix(p, st).toarray()
    B = hamiltonian_matrix_vec(p, st).toarray()
    assert np.array_equal(A, B)
    q = I.heisenberg_square(4)
    st = basis(16, 8, 8, True)[:300]
    A = hamiltonian_matrix(q, st).toarray()
    B = hamiltonian_matrix_vec(q, st).toarray()
    assert np.array_equal(A, B)


def test_singlet_exchange_sign():
    """Two-site Heisenberg singlet (f symmetric, N = 1): E_loc = -3J/4 on
    both configurations (fermion sign of S+S- in the labelled basis)."""
    lat = I.Lattice(2, 1)
    p = I.make_problem("s2", I.chain(4, 1), 2, t=0.0, J1=1.0, local_spin=True,
                       gutzwiller=False, f_full=True, noise=0.0, f_init="none")
    p = p.copy_with(lat=lat, ex_i=np.array([0], np.int32), ex_j=np.array([1], np.int32),
                    ex_J=np.array([1.0]), U=np.zeros(2), f_idx=np.array([-1, 0, 0, -1], np.int32),
                    f_sign=np.ones(4, np.int8), n_f=1, params=np.array([0.7]),
                    g_idx=np.full(2, -1, np.int32), n_g=0, v_idx=np.full(4, -1, np.int32), n_v=0)
    wf = Wavefunction(p)
    for ele in ([0, 1], [1, 0]):
        assert local_energy(wf, fock.from_labels(ele, 2)) == pytest.approx(-0.75, abs=1e-14)


# --------------------------------------------------------------------------
# Free-fermion limit (Appendix B): U = 0 pairing state has zero variance
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name,build,L,bc,N", [
    ("ring8", lambda: I.ring8_hubbard(noise=0.0, U=0.0), (8, 1), (1, 1), 4),
    ("square8", lambda: I.square8_hubbard(noise=0.0, U=0.0), (8, 8), (1, -1), 32),
])
def test_free_fermion_zero_variance(name, build, L, bc, N):
    p = build()
    wf = Wavefunction(p)
    e0 = free_fermion_energy(L[0], L[1], bc[0], bc[1], N)
    if name == "ring8":
        assert e0 == pytest.approx(-9.656854249492381, abs=1e-12)
    cfg = I.initial_configs(p.Ns, p.Ne, 12, False, 5)
    checked = 0
    for c in cfg:
        n = fock.from_labels(c, p.Ns)
        X, _ = wf.X(n)
        if np.linalg.cond(X) > 1e8:     # a node of the Slater state: roundoff amplitude
            continue
        assert local_energy(wf, n) == pytest.approx(e0, abs=1e-8)
        checked += 1
        if checked >= 3:
            break
    assert checked >= 2


def test_free_fermion_closed_shell_energies():
    """Shell closures used by the workloads (textbook sums)."""
    assert free_fermion_energy(8, 8, 1, -1, 32) / 64 == pytest.approx(-1.64213, abs=1e-5)
    assert free_fermion_energy(16, 16, -1, -1, 112) / 256 == pytest.approx(-1.61058, abs=1e-5)


def test_apbc_sublattice_sign_example():
    """Appendix A: 4-site anti-periodic chain, 2-site sublattice: f_03 = -f_21."""
    line = [l for l in open(os.path.join(GOLD, "apbc_example.txt")) if not l.startswith("#")][0]
    L, bc, Wsub, i, j, k, l, rel = (int(x) for x in line.split())
    f_idx, f_sign, n_f = I.sublattice_f_layout(I.chain(L, bc), Wsub, 1)
    f_idx = f_idx.reshape(L, L)
    f_sign = f_sign.reshape(L, L)
    assert f_idx[i, j] == f_idx[k, l]
    assert f_sign[k, l] * f_sign[i, j] == rel
    assert n_f == Wsub * L


# --------------------------------------------------------------------------
# Derivatives, variational bound, estimator, SR
# --------------------------------------------------------------------------
def test_log_derivatives_match_finite_differences():
    p = I.make_problem("r6", I.chain(6, -1), 6, U=4.0, sub=(2, 1), jastrow="chain",
                       noise=0.2, seed=4)
    p.params[:3] = [-0.4, 0.3, -0.1]
    wf = Wavefunction(p)
    for c in I.initial_configs(6, 6, 3, False, 9):
        n = fock.from_labels(c, 6)
        a = wf.log_derivatives(n)
        b = wf.log_derivatives_fd(n, 1e-6)
        assert np.allclose(a, b, rtol=1e-6, atol=1e-7)


def test_log_derivatives_full_f_heisenberg():
    p = I.heisenberg_square(2 * 2, noise=0.3, seed=2, sub=(4, 4))
    wf = Wavefunction(p)
    c = I.initial_configs(16, 16, 1, True, 1)[0]
    n = fock.from_labels(c, 16)
    a = wf.log_derivatives(n)
    idx = np.nonzero(a)[0][:12]
    for k in idx:
        pp, pm = p.params.copy(), p.params.copy()
        pp[k] += 1e-6
        pm[k] -= 1e-6
        fd = (Wavefunction(p, pp).amplitude_slog(n)[1] - Wavefunction(p, pm).amplitude_slog(n)[1]) / 2e-6
        assert a[k] == pytest.approx(fd, rel=1e-5, abs=1e-7)


def test_variational_bound_and_exact_sr():
    p = I.make_problem("r6", I.chain(6, -1), 6, U=4.0, sub=(2, 1), jastrow="chain",
                       noise=0.2, seed=4)
    e_ed = ground_state_energy(p)
    rng = np.random.default_rng(0)
    for _ in range(3):
        params = p.params + rng.normal(0, 0.1, p.params.size)
        ex = enumerate_expectations(Wavefunction(p, params))
        assert ex["energy"] >= e_ed - 1e-12
        assert np.linalg.eigvalsh(ex["S"]).min() > -1e-12


def test_metropolis_matches_enumeration():
    """MC energy within 3 standard errors of the exact expectation (Eq. MC)."""
    p = I.make_problem("r4", I.chain(4, -1), 4, U=4.0, sub=(2, 1), jastrow="chain",
                       noise=0.3, seed=8, p_exchange=0.5)
    p.params[0] = -0.5
    wf = Wavefunction(p)
    ex = enumerate_expectations(wf)
    ele0 = I.initial_configs(4, 4, 8, False, 3)
    res = run_sampling(wf, ele0, seed=17, system=0, n_warmup=5, n_samples=100,
                       sweeps_between=2, p_exchange=0.5)
    E = res["E"].reshape(8, 100)
    walker_means = E.mean(axis=1)
    se = walker_means.std(ddof=1) / math.sqrt(8)
    assert abs(E.mean() - ex["energy"]) < 3 * se + 1e-12
    # O averages too.
    O = res["O"].reshape(8, 100, -1).mean(axis=1)
    se_o = O.std(axis=0, ddof=1) / math.sqrt(8)
    assert np.all(np.abs(O.mean(axis=0) - ex["obar"]) < 3 * se_o + 1e-3)


def test_local_spin_moves_keep_single_occupancy():
    p = I.heisenberg_square(4, noise=0.2, seed=1)
    wf = Wavefunction(p)
    ele0 = I.initial_configs(16, 16, 1, True, 2)
    res = run_sampling(wf, ele0, 3, 0, 2, 0, 1, 1.0, measure=False)
    assert sorted(res["ele"][0]) == list(range(16))
    assert res["n_acc"] > 0


def test_sr_cholesky_and_cg_agree():
    E, O = I.random_samples(500, 40, seed=3)
    d1, info = sr_step(E, O, 0.05, shift_rel=1e-3, solver="cholesky")
    d2, info2 = sr_step(E, O, 0.05, shift_rel=1e-3, solver="cg", cg_eps=1e-13)
    assert np.allclose(d1, d2, rtol=1e-10, atol=1e-13)
    assert 0 < info2["cg_iters"] <= 40


def test_sr_matrices_definition():
    """S and g against sums over samples written out per entry."""
    E, O = I.random_samples(50, 5, seed=4)
    S, g, obar, ebar = sr_matrices(E, O)
    for k in range(5):
        for m in range(5):
            ref = sum(O[u, k] * O[u, m] for u in range(50)) / 50 - (sum(O[:, k]) / 50) * (sum(O[:, m]) / 50)
            assert S[k, m] == pytest.approx(ref, rel=1e-12, abs=1e-14)
        refg = sum(E[u] * O[u, k] for u in range(50)) / 50 - (sum(E) / 50) * (sum(O[:, k]) / 50)
        assert g[k] == pytest.approx(refg, rel=1e-12, abs=1e-14)


def test_srcg_matvec_equals_dense():
    E, O = I.random_samples(200, 30, seed=5)
    S, g, obar, _ = sr_matrices(E, O)
    v = np.random.default_rng(1).standard_normal(30)
    St = shifted(S, 1e-3, 1e-4)
    assert np.allclose(srcg_matvec(O, obar, np.diag(S), v, 1e-3, 1e-4), St @ v, rtol=1e-12, atol=1e-13)


def test_cg_solves_spd_system():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((30, 30))
    A = A @ A.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    x, it = cg(lambda v: A @ v, b, eps=1e-14)
    assert np.allclose(A @ x, b, atol=1e-10)
    assert np.allclose(solve_cholesky(A, b), x, atol=1e-10)


def test_mlp_factor_derivatives_and_limit():
    """MLP correlation factor: analytic O_k against finite differences, and
    w2 = b2 = 0 reduces psi to the plain projected Pfaffian."""
    p = I.make_problem("r6m", I.chain(6, -1), 6, U=4.0, sub=(2, 1), jastrow="chain",
                       noise=0.2, seed=4, mlp_hidden=3, mlp_std=0.3)
    wf = Wavefunction(p)
    c = I.initial_configs(6, 6, 1, False, 9)[0]
    n = fock.from_labels(c, 6)
    a = wf.log_derivatives(n)
    b = wf.log_derivatives_fd(n, 1e-6)
    assert np.allclose(a, b, rtol=1e-6, atol=1e-7)
    q = p.params.copy()
    base = p.n_g + p.n_v + p.n_f + 3 * 12
    q[base + 3:] = 0.0                      # w2 = 0, b2 = 0
    plain = p.copy_with(n_hidden=0, params=p.params[:p.n_g + p.n_v + p.n_f])
    assert Wavefunction(p, q).amplitude_slog(n)[1] == pytest.approx(
        Wavefunction(plain).amplitude_slog(n)[1], rel=1e-14)
