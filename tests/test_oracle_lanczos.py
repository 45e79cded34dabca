"""Pins of the first-step power-Lanczos oracle (oracle.lanczos, Sec. 3.4):
with the exact rho(x) the four moments are <H>, <H^2> (twice) and <H^3> of
the state vector, computed here by matrix powers of H; E_1(alpha) from the
moments is the Rayleigh quotient of (1 + alpha H) psi; the quadratic's root
minimises E_1, lies below <H> and above the ground state; an eigenstate
gives h_k = E^k and alpha-independent E_1.  No GPU.
"""
import math

import numpy as np
import pytest

from oracle import fock
from oracle.hamiltonian import basis, hamiltonian_matrix_vec
from oracle.lanczos import (energy, exact_moments, local_f, moments_from_local, optimal_alpha,
                            sampled_moments)
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I


def systems():
    hub = I.make_problem("c6", I.chain(6, -1), 4, U=3.0, f_full=True, jastrow="chain",
                         f_init="none", noise=0.6, seed=9)
    hub.params[:3] = [-0.4, 0.2, -0.1]
    heis = I.make_problem("h6", I.chain(6, 1), 6, t=0.0, J1=1.0, local_spin=True, f_full=True,
                          gutzwiller=False, noise=0.3, seed=4)
    return {"hubbard_chain6": hub, "heisenberg_ring6": heis}


def state_vector(wf, p):
    st = basis(p.Ns, p.Ne // 2, p.Ne // 2, p.local_spin)
    v = np.array([wf.amplitude(n) for n in st])
    H = hamiltonian_matrix_vec(p, st).toarray()
    return v / np.linalg.norm(v), H


@pytest.mark.parametrize("name", ["hubbard_chain6", "heisenberg_ring6"])
def test_exact_moments_are_matrix_moments(name):
    p = systems()[name]
    wf = Wavefunction(p)
    h = exact_moments(wf)
    v, H = state_vector(wf, p)
    Hv = H @ v
    assert h["h1"] == pytest.approx(v @ Hv, rel=1e-11)
    assert h["h2_11"] == pytest.approx(Hv @ Hv, rel=1e-11)
    assert h["h2_20"] == pytest.approx(Hv @ Hv, rel=1e-11)
    assert h["h3_12"] == pytest.approx(Hv @ (H @ Hv), rel=1e-11)


@pytest.mark.parametrize("name", ["hubbard_chain6", "heisenberg_ring6"])
def test_first_step_energy_and_optimum(name):
    p = systems()[name]
    wf = Wavefunction(p)
    h = exact_moments(wf)
    v, H = state_vector(wf, p)
    for alpha in (-0.3, -0.05, 0.1):
        u = v + alpha * (H @ v)
        assert energy(h, alpha) == pytest.approx(u @ H @ u / (u @ u), rel=1e-10)
    a_opt, e_opt = optimal_alpha(h)
    grid = np.linspace(a_opt - 0.5, a_opt + 0.5, 2001)
    assert e_opt <= min(energy(h, t) for t in grid) + 1e-12
    e0 = np.linalg.eigvalsh(H)[0]
    assert e0 - 1e-10 <= e_opt < h["h1"]


def test_eigenstate_moments():
    """Two-site Heisenberg singlet (an eigenstate, E = -3/4): h_k = E^k and
    E_1 = E for every alpha."""
    p = I.make_problem("s2", I.chain(4, 1), 2, t=0.0, J1=1.0, local_spin=True,
                       gutzwiller=False, f_full=True, noise=0.0, f_init="none")
    p = p.copy_with(lat=I.Lattice(2, 1), ex_i=np.array([0], np.int32), ex_j=np.array([1], np.int32),
                    ex_J=np.array([1.0]), U=np.zeros(2), f_idx=np.array([-1, 0, 0, -1], np.int32),
                    f_sign=np.ones(4, np.int8), n_f=1, params=np.array([0.7]),
                    g_idx=np.full(2, -1, np.int32), n_g=0, v_idx=np.full(4, -1, np.int32), n_v=0)
    wf = Wavefunction(p)
    for ele in ([0, 1], [1, 0]):
        fh, fh2 = local_f(wf, fock.from_labels(ele, 2))
        assert fh == pytest.approx(-0.75, abs=1e-14)
        assert fh2 == pytest.approx(0.5625, abs=1e-14)
    h = exact_moments(wf)
    for alpha in (-1.0, 0.0, 0.4):
        assert energy(h, alpha) == pytest.approx(-0.75, abs=1e-12)


def test_sampled_moments_are_means_of_local_values():
    p = systems()["hubbard_chain6"]
    wf = Wavefunction(p)
    cfgs = [fock.from_labels(e, p.Ns) for e in I.initial_configs(p.Ns, p.Ne, 4, False, 5)]
    h = sampled_moments(wf, cfgs)
    vals = [local_f(wf, n) for n in cfgs]
    ref = moments_from_local([v[0] for v in vals], [v[1] for v in vals])
    for k in ref:
        assert h[k] == pytest.approx(ref[k], rel=1e-14)
    fh = np.array([v[0] for v in vals])
    fh2 = np.array([v[1] for v in vals])
    assert h["h1"] == pytest.approx(fh.mean(), rel=1e-14)
    assert h["h2_11"] == pytest.approx((fh * fh).mean(), rel=1e-14)
    assert h["h2_20"] == pytest.approx(fh2.mean(), rel=1e-14)
    assert h["h3_12"] == pytest.approx((fh * fh2).mean(), rel=1e-14)


@pytest.mark.parametrize("name", ["hubbard_chain6", "heisenberg_ring6"])
def test_local_values_are_matrix_ratios(name):
    """F(x, H) = (H v)_x / v_x and F(x, H^2) = (H^2 v)_x / v_x on every
    configuration (the moments with the exact rho cannot tell
    <F(x,H)^2> from <F(x,H^2)>; the local values can)."""
    p = systems()[name]
    wf = Wavefunction(p)
    st = basis(p.Ns, p.Ne // 2, p.Ne // 2, p.local_spin)
    v, H = state_vector(wf, p)
    Hv, H2v = H @ v, H @ (H @ v)
    for k in range(0, len(st), 7):
        if abs(v[k]) < 1e-8:
            continue
        fh, fh2 = local_f(wf, st[k])
        assert fh == pytest.approx(Hv[k] / v[k], rel=1e-9, abs=1e-9)
        assert fh2 == pytest.approx(H2v[k] / v[k], rel=1e-9, abs=1e-9)
