"""Exact enumeration over all configurations of a tiny system: the
expectation values that the Monte Carlo estimator of Eq. MC approximates,
with rho(x) = |<x|psi>|^2 / <psi|psi> (Sec. 3.1.1), and the exact SR
matrices for the current parameters."""
import numpy as np

from .hamiltonian import basis, local_energy
from .sr import sr_matrices


def enumerate_expectations(wf):
    N = wf.Ne // 2
    states = basis(wf.Ns, N, N, wf.local_spin, wf.local_sites)
    amps = np.array([wf.amplitude(n) for n in states])
    w = amps ** 2
    keep = w > 0
    states = [s for s, k in zip(states, keep) if k]
    w = w[keep] / w[keep].sum()
    E = np.array([local_energy(wf, n) for n in states])
    O = np.array([wf.log_derivatives(n) for n in states])
    S, g, obar, energy = sr_matrices(E, O, w)
    var = float(w @ (E - energy) ** 2)
    return dict(energy=energy, variance=var, S=S, g=g, obar=obar,
                states=states, weights=w, E=E, O=O)
