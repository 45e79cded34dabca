"""Pins of the oracle's SR matrices (Sec. 3.3.1, Eq. SR_equation_system)
against what the mathematics fixes, independently of the formula itself.

For real parameters and a real wave function, with rho(x) = psi(x)^2 /
<psi|psi> and O_k = d ln psi / d alpha_k:

* the force is half the gradient of the variational energy,
  g_k = <E_loc O_k> - <E_loc><O_k> = (1/2) dE/dalpha_k,
  E(alpha) = <psi|H|psi> / <psi|psi>;
* S is the metric of the normalised state: for a displacement t*delta,
  1 - |<psi(a)|psi(a + t delta)>|^2 / (|psi(a)|^2 |psi(a + t delta)|^2)
  = t^2 delta^T S delta + O(t^3);
* hence a small SR step alpha -> alpha - dtau S~^-1 g lowers E, by
  2 dtau g^T S~^-1 g to first order in dtau.

E(alpha) comes from the Hamiltonian matrix and the amplitude vector over the
whole basis (a Rayleigh quotient, not the local-energy routine), and the
overlaps from the amplitude vectors alone; S and g come from
`oracle.sr.sr_matrices` on exactly enumerated (E_loc, O) rows with weights
rho.  Three planted mistakes (a force without the <E><O> term, a force twice
too large, an uncentred S) each fail a pin.
"""
import numpy as np
import pytest

from oracle.exact import enumerate_expectations
from oracle.hamiltonian import basis, hamiltonian_matrix_vec
from oracle.sr import shifted, solve_cholesky, sr_matrices
from oracle.wavefunction import Wavefunction
from paper_1711_11418_gb300 import inputs as I


def _ring6_hubbard():
    p = I.make_problem("r6", I.chain(6, -1), 6, U=4.0, sub=(2, 1), jastrow="chain",
                       noise=0.2, seed=4)
    p.params[0] = -0.4            # Gutzwiller: <O_g> = <D> is far from 0
    p.params[1:3] = [0.15, -0.1]  # Jastrow
    return p


def _ring4_heisenberg():
    return I.make_problem("h4", I.chain(4, 1), 4, t=0.0, J1=1.0, local_spin=True,
                          f_full=True, gutzwiller=False, noise=0.3, seed=6)


def _ring4_hubbard_mlp():
    return I.make_problem("r4m", I.chain(4, -1), 4, U=3.0, sub=(2, 1), jastrow="chain",
                          noise=0.2, seed=2, mlp_hidden=2, mlp_std=0.3)


MODELS = {"ring6_hubbard": _ring6_hubbard, "ring4_heisenberg": _ring4_heisenberg,
          "ring4_hubbard_mlp": _ring4_hubbard_mlp}


class Exact:
    """Amplitude vectors and the Rayleigh quotient over the whole basis."""

    def __init__(self, prob):
        self.prob = prob
        self.states = basis(prob.Ns, prob.N, prob.N, prob.local_spin,
                            getattr(prob, "local_sites", None))
        self.H = hamiltonian_matrix_vec(prob, self.states)

    def psi(self, params):
        wf = Wavefunction(self.prob, params)
        return np.array([wf.amplitude(n) for n in self.states])

    def energy(self, params):
        v = self.psi(params)
        return float(v @ (self.H @ v) / (v @ v))

    def infidelity(self, a, b):
        va, vb = self.psi(a), self.psi(b)
        return 1.0 - (va @ vb) ** 2 / ((va @ va) * (vb @ vb))


def exact_rows(prob, params):
    ex = enumerate_expectations(Wavefunction(prob, params))
    return ex["E"], ex["O"], ex["weights"]


def force_pin_error(srm, prob, h=1e-5):
    """max_k |g_k - (1/2) dE/dalpha_k| relative to max |g|, central differences."""
    X = Exact(prob)
    a = prob.params.copy()
    _, g, _, _ = srm(*exact_rows(prob, a))
    fd = np.empty(a.size)
    for k in range(a.size):
        ap, am = a.copy(), a.copy()
        ap[k] += h
        am[k] -= h
        fd[k] = 0.5 * (X.energy(ap) - X.energy(am)) / (2 * h)
    return np.max(np.abs(g - fd)) / np.max(np.abs(fd)), g, fd


def metric_pin_error(srm, prob, n_dirs=3, t=2e-4, seed=0):
    """max over random directions of |delta^T S delta - c2| / c2, with c2 the
    second-order coefficient of the infidelity (odd orders cancelled by +-t)."""
    X = Exact(prob)
    a = prob.params.copy()
    S, _, _, _ = srm(*exact_rows(prob, a))
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(n_dirs):
        d = rng.standard_normal(a.size)
        d /= np.linalg.norm(d)
        c2 = 0.5 * (X.infidelity(a, a + t * d) + X.infidelity(a, a - t * d)) / t ** 2
        worst = max(worst, abs(d @ S @ d - c2) / c2)
    return worst


@pytest.mark.parametrize("name", sorted(MODELS))
def test_force_is_half_the_energy_gradient(name):
    err, g, fd = force_pin_error(sr_matrices, MODELS[name]())
    assert np.max(np.abs(fd)) > 1e-3          # a state away from a stationary point
    assert err < 1e-7, err


@pytest.mark.parametrize("name", sorted(MODELS))
def test_metric_is_the_overlap_curvature(name):
    assert metric_pin_error(sr_matrices, MODELS[name]()) < 1e-5


@pytest.mark.parametrize("name", sorted(MODELS))
def test_exact_sr_step_lowers_the_energy(name):
    prob = MODELS[name]()
    X = Exact(prob)
    a = prob.params.copy()
    S, g, _, _ = sr_matrices(*exact_rows(prob, a))
    x = solve_cholesky(shifted(S, 1e-3, 1e-6), g)
    e0 = X.energy(a)
    pred = 2.0 * g @ x                          # first-order decrease per unit dtau
    assert pred > 0
    for dtau in (0.02, 0.01):
        e1 = X.energy(a - dtau * x)
        assert e1 < e0
        # first order in dtau: the relative gap shrinks with dtau
        assert abs((e0 - e1) / (dtau * pred) - 1.0) < 50 * dtau


def test_uniform_samples_equal_weighted_rows():
    """Rows repeated m_u times give the weights m_u / sum m (plain sample mean)."""
    rng = np.random.default_rng(3)
    E, O = rng.standard_normal(7), rng.standard_normal((7, 4))
    m = np.array([1, 3, 2, 1, 4, 1, 2])
    Er, Or = np.repeat(E, m), np.repeat(O, m, axis=0)
    for a, b in zip(sr_matrices(Er, Or), sr_matrices(E, O, m.astype(float))):
        assert np.allclose(a, b, rtol=1e-13, atol=1e-14)


# --------------------------------------------------------------------------
# Planted mistakes (in the oracle's formula, on the CPU): each fails a pin.
# --------------------------------------------------------------------------
def _force_without_mean_term(E, O, weights=None):
    S, g, obar, ebar = sr_matrices(E, O, weights)
    return S, g + ebar * obar, obar, ebar          # g = <E O> only


def _uncentred_metric(E, O, weights=None):
    S, g, obar, ebar = sr_matrices(E, O, weights)
    return S + np.outer(obar, obar), g, obar, ebar  # S = <O O^T> only


def _force_times_two(E, O, weights=None):
    S, g, obar, ebar = sr_matrices(E, O, weights)
    return S, 2.0 * g, obar, ebar                   # dE/dalpha instead of half of it


def test_planted_mistakes_fail_the_pins():
    prob = _ring6_hubbard()
    assert force_pin_error(_force_without_mean_term, prob)[0] > 0.1
    assert force_pin_error(_force_times_two, prob)[0] > 0.5
    assert metric_pin_error(_uncentred_metric, prob) > 0.1
