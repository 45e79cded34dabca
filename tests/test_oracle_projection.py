"""Pins of the projection oracle (oracle.projection; Sec. 3.2.2, Eqs. momP
and pointP).  Each symmetry operation is also built here as a many-body
matrix in the canonical basis, from its forward map applied with the
operator algebra (the oracle maps configurations backwards), and checked:

* the translations form the group (T_R1 T_R2 = T_{R1+R2}) and commute with
  H, including the anti-periodic boundary signs (App. A); so do the point
  operations of a 3x3 square lattice that are symmetries;
* <x|L|phi> of the oracle equals (sum_g w_g T_g phi)_x of the matrices;
* L_K phi is a momentum eigenstate, T_R L_K = exp(-i K.R) L_K;
* completeness: sum over all K of L_K phi = phi;
* the U = 0 closed-shell pairing state has total momentum 0;
* the projected energy by local estimators (Eq. MC) equals the Rayleigh
  quotient of the projected vector and lies above the ground state of its
  momentum sector.  No GPU.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import fock
from oracle.hamiltonian import basis, hamiltonian_matrix_vec, local_energy
from oracle.projection import (ProjectedWavefunction, combine, momentum_weights, point_ops,
                               projected_pair_amplitude, translations, pair_amplitude_slog)
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I


def op_matrix(op, states, Ns):
    """Many-body matrix of T_g: T_g |x> = prod_k s(r_k) c^dag_{g(r_k)} |0>."""
    index = {s: k for k, s in enumerate(states)}
    M = np.zeros((len(states), len(states)))
    for col, n in enumerate(states):
        coef = 1.0
        string = []
        for I_ in fock.occupied(n, 2 * Ns):
            spin, site = (1, I_ - Ns) if I_ >= Ns else (0, I_)
            coef *= op.sign[site]
            string.append(("+", int(op.perm[site]) + Ns * spin))
        r = fock.apply_string(string, (coef, 0))
        M[index[r[1]], col] = r[0]
    return M


def pair_vector(wf, states):
    out = np.zeros(len(states))
    for k, n in enumerate(states):
        s, l = pair_amplitude_slog(wf, n)
        out[k] = s * math.exp(l) if s != 0.0 else 0.0
    return out


def chain6():
    p = I.make_problem("c6", I.chain(6, -1), 4, U=3.0, f_full=True, jastrow="chain",
                       f_init="none", noise=0.6, seed=9)
    p.params[:3] = [-0.4, 0.2, -0.1]
    return p


def test_translations_form_the_group_and_commute_with_H():
    p = chain6()
    st = basis(p.Ns, 2, 2)
    H = hamiltonian_matrix_vec(p, st).toarray()
    tr = translations(p.lat)
    Ms = {R: op_matrix(op, st, p.Ns) for op, R in tr}
    for (_, R1) in tr:
        for (_, R2) in tr:
            R = ((R1[0] + R2[0]) % p.lat.Lx, 0)
            np.testing.assert_allclose(Ms[R1] @ Ms[R2], Ms[R], atol=1e-14)
        np.testing.assert_allclose(H @ Ms[R1], Ms[R1] @ H, atol=1e-12)


def test_point_operations_of_a_square_lattice():
    """3x3, anti-periodic in x and y, Ne = 4: the operations that commute
    with H compose like the point group with the translations."""
    lat = I.square(3, 3, -1, -1)
    p = I.make_problem("s3", lat, 4, U=2.0, sub=(1, 1), f_full=True, f_init="none",
                       noise=0.5, seed=2)
    st = basis(p.Ns, 2, 2)
    H = hamiltonian_matrix_vec(p, st).toarray()
    sym = []
    for op, name in point_ops(lat):
        M = op_matrix(op, st, p.Ns)
        if np.allclose(H @ M, M @ H, atol=1e-12):
            sym.append((op, M, name))
    names = {n for _, _, n in sym}
    assert {"E", "C2", "Mx", "My"} <= names          # the rectangle group at least
    for a, Ma, _ in sym:
        for b, Mb, _ in sym:
            np.testing.assert_allclose(op_matrix(a.compose(b), st, p.Ns), Ma @ Mb, atol=1e-14)


@pytest.mark.parametrize("m", [0, 1, 3])
def test_projected_amplitude_equals_matrix_route(m):
    p = chain6()
    wf = Wavefunction(p)
    st = basis(p.Ns, 2, 2)
    tr = translations(p.lat)
    K = (2 * math.pi * m / p.lat.Lx, 0.0)
    W = momentum_weights(tr, K)
    phi = pair_vector(wf, st)
    Lphi = sum(w * (op_matrix(op, st, p.Ns) @ phi) for op, w in W)
    v = np.array([projected_pair_amplitude(wf, n, W) for n in st])
    np.testing.assert_allclose(v, Lphi, atol=1e-12)
    # momentum eigenstate: T_R L_K phi = exp(-i K.R) L_K phi
    for op, R in tr:
        np.testing.assert_allclose(op_matrix(op, st, p.Ns) @ v,
                                   cmath.exp(-1j * K[0] * R[0]) * v, atol=1e-12)


def test_completeness_over_momenta():
    p = chain6()
    wf = Wavefunction(p)
    tr = translations(p.lat)
    st = basis(p.Ns, 2, 2)
    tot = np.zeros(len(st), complex)
    for m in range(p.lat.Lx):
        W = momentum_weights(tr, (2 * math.pi * m / p.lat.Lx, 0.0))
        tot += np.array([projected_pair_amplitude(wf, n, W) for n in st])
    np.testing.assert_allclose(tot, pair_vector(wf, st), atol=1e-12)


def test_closed_shell_pairing_state_has_zero_momentum():
    """U = 0 pairing of the lowest orbitals of the anti-periodic 6-ring
    (closed shell, pairs k, -k): L_0 phi = phi, L_K phi = 0 for K != 0."""
    p = I.make_problem("ff6", I.chain(6, -1), 4, U=0.0, f_full=True, gutzwiller=False,
                       noise=0.0)
    wf = Wavefunction(p)
    st = basis(p.Ns, 2, 2)
    phi = pair_vector(wf, st)
    tr = translations(p.lat)
    for m in range(6):
        W = momentum_weights(tr, (2 * math.pi * m / 6, 0.0))
        v = np.array([projected_pair_amplitude(wf, n, W) for n in st])
        np.testing.assert_allclose(v, phi if m == 0 else 0 * phi, atol=1e-12)


@pytest.mark.parametrize("m", [0, 3])
def test_projected_energy_two_routes_and_bound(m):
    """Real characters (K = 0, pi): E from the local estimators of Eq. MC
    weighted by rho(x) equals v^T H v / v^T v of the projected vector
    (correlation factors included), and is >= the lowest eigenvalue of H in
    that momentum sector."""
    p = chain6()
    wf = Wavefunction(p)
    tr = translations(p.lat)
    W = [(op, complex(w).real) for op, w in momentum_weights(tr, (math.pi * m / 3, 0.0))]
    pwf = ProjectedWavefunction(wf, W)
    st = basis(p.Ns, 2, 2)
    amps = np.array([pwf.amplitude(n) for n in st])
    keep = amps != 0
    rho = amps[keep] ** 2 / np.sum(amps[keep] ** 2)
    e_mc = float(sum(r * local_energy(pwf, n) for r, n, k in
                     zip(rho, [s for s, k in zip(st, keep) if k], range(len(rho)))))
    H = hamiltonian_matrix_vec(p, st).toarray()
    e_rq = float(amps @ H @ amps / (amps @ amps))
    assert e_mc == pytest.approx(e_rq, rel=1e-11, abs=1e-11)
    # lowest eigenvalue within the sector: H on the range of the projector L_K
    Pk = sum(w * op_matrix(op, st, p.Ns) for op, w in W)
    pw, pv = np.linalg.eigh(0.5 * (Pk + Pk.T))
    Q = pv[:, pw > 0.5]
    assert Q.shape[1] > 0
    e_sector = np.linalg.eigvalsh(Q.T @ H @ Q)[0]
    assert e_rq >= e_sector - 1e-10


def test_combined_momentum_and_point_group_projection():
    """L = L_K L_P on the 3x3 lattice (K = 0, A1: every character 1): the
    oracle's amplitudes equal the matrix route, and the projected state is
    invariant under every translation and point operation."""
    lat = I.square(3, 3, -1, -1)
    p = I.make_problem("s3", lat, 4, U=2.0, sub=(1, 1), f_full=True, f_init="none",
                       noise=0.5, seed=2)
    wf = Wavefunction(p)
    st = basis(p.Ns, 2, 2)
    tr = translations(lat)
    pts = point_ops(lat)
    W = combine(momentum_weights(tr, (0.0, 0.0)), [(op, 1.0 / len(pts)) for op, _ in pts])
    phi = pair_vector(wf, st)
    Mphi = sum(w * (op_matrix(op, st, p.Ns) @ phi) for op, w in W)
    v = np.array([projected_pair_amplitude(wf, n, W) for n in st])
    np.testing.assert_allclose(v, Mphi, atol=1e-12)
    assert np.linalg.norm(v) > 1e-3
    for op, _ in tr + pts:
        np.testing.assert_allclose(op_matrix(op, st, p.Ns) @ v, v, atol=1e-12)


@pytest.mark.parametrize("m", ["K0", "Kpi"])
def test_projected_log_derivatives_match_finite_differences(m):
    """O_k of the projected state (Sec. 3.3.1 applied to psi = P <x|L|phi>)
    against central differences of ln|psi(x)| with perturbed parameters."""
    p = chain6()
    K = (0.0, 0.0) if m == "K0" else (math.pi, 0.0)
    ops = momentum_weights(translations(p.lat), K)
    ops = [(op, complex(w).real) for op, w in ops]
    wf = Wavefunction(p)
    pw = ProjectedWavefunction(wf, ops)
    h = 1e-6
    checked = 0
    for n in basis(p.Ns, 2, 2)[::7]:
        s0, _ = pw.amplitude_slog(n)
        if s0 == 0.0:
            continue
        a = pw.log_derivatives(n)
        fd = np.zeros_like(a)
        for k in range(a.size):
            pp, pm = p.params.copy(), p.params.copy()
            pp[k] += h
            pm[k] -= h
            lp = ProjectedWavefunction(Wavefunction(p, pp), ops).amplitude_slog(n)[1]
            lm = ProjectedWavefunction(Wavefunction(p, pm), ops).amplitude_slog(n)[1]
            fd[k] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(a, fd, rtol=1e-5, atol=1e-6)
        checked += 1
    assert checked >= 5
