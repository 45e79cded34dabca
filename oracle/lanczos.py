"""First-step power-Lanczos (Sec. 3.4): |psi_1> = (1 + alpha_1 H)|psi>,

    E_1(alpha) = (h1 + alpha (h2(20) + h2(11)) + alpha^2 h3(12))
                 / (1 + 2 alpha h1 + alpha^2 h2(11)),

with the moments averaged over configurations drawn from rho(x):
h1 = <F(x,H)>, h2(11) = <F(x,H) F(x,H)>, h2(20) = <F(x,H^2)>,
h3(12) = <F(x,H) F(x,H^2)>, F(x, A) = <x|A|psi> / <x|psi> (real psi and H).
alpha_1 is the minimising root of dE_1/dalpha = 0, a quadratic equation.

Test infrastructure, like the rest of ``oracle``.

F(x, H^2) = sum_x' <x|H|x'> (H psi)(x') / psi(x) with (H psi)(x') =
sum_x'' <x'|H|x''> psi(x''): every amplitude from scratch, and no division
by psi(x'), which may vanish where (H psi)(x') does not.
"""
import math

import numpy as np

from .hamiltonian import apply_H, basis


class _Amplitudes:
    def __init__(self, wf):
        self.wf = wf
        self.cache = {}

    def __call__(self, n):
        if n not in self.cache:
            self.cache[n] = self.wf.amplitude(n)
        return self.cache[n]


def _h_psi(wf, amp, n):
    """(H psi)(x) = sum_x' <x|H|x'> psi(x') (H real symmetric)."""
    return sum(coef * amp(n2) for n2, coef in apply_H(wf.prob, n).items())


def local_f(wf, n, amp=None):
    """(F(x, H), F(x, H^2)) of one configuration."""
    amp = amp or _Amplitudes(wf)
    a0 = amp(n)
    if a0 == 0.0:
        raise ZeroDivisionError("psi(x) = 0")
    fh = _h_psi(wf, amp, n) / a0
    fh2 = sum(coef * _h_psi(wf, amp, n2) for n2, coef in apply_H(wf.prob, n).items()) / a0
    return fh, fh2


def moments_from_local(fh, fh2, weights=None):
    """h1, h2(11), h2(20), h3(12) as (weighted) means of the local values."""
    fh = np.asarray(fh, np.float64)
    fh2 = np.asarray(fh2, np.float64)
    w = np.full(fh.size, 1.0 / fh.size) if weights is None else np.asarray(weights, np.float64)
    return dict(h1=float(w @ fh), h2_11=float(w @ (fh * fh)), h2_20=float(w @ fh2),
                h3_12=float(w @ (fh * fh2)))


def sampled_moments(wf, configs):
    """The moments over configurations drawn from rho(x) (the Monte Carlo
    estimate of Sec. 3.4)."""
    amp = _Amplitudes(wf)
    vals = [local_f(wf, n, amp) for n in configs]
    return moments_from_local([v[0] for v in vals], [v[1] for v in vals])


def exact_moments(wf):
    """The moments with the exact rho(x), by enumeration (tiny systems)."""
    N = wf.Ne // 2
    states = basis(wf.Ns, N, N, wf.local_spin, getattr(wf, "local_sites", None))
    amp = _Amplitudes(wf)
    a = np.array([amp(n) for n in states])
    keep = np.nonzero(a != 0.0)[0]
    rho = a[keep] ** 2 / np.sum(a[keep] ** 2)
    vals = [local_f(wf, states[k], amp) for k in keep]
    return moments_from_local([v[0] for v in vals], [v[1] for v in vals], rho)


def energy(h, alpha):
    """E_1(alpha) of Sec. 3.4 from the moments."""
    num = h["h1"] + alpha * (h["h2_20"] + h["h2_11"]) + alpha * alpha * h["h3_12"]
    den = 1.0 + 2.0 * alpha * h["h1"] + alpha * alpha * h["h2_11"]
    return num / den


def optimal_alpha(h):
    """The root of dE_1/dalpha = 0 with the lower E_1: with
    E_1 = (a + b t + c t^2) / (1 + d t + e t^2) the condition is
    (b - a d) + 2 (c - a e) t + (c d - b e) t^2 = 0."""
    a, b, c = h["h1"], h["h2_20"] + h["h2_11"], h["h3_12"]
    d, e = 2.0 * h["h1"], h["h2_11"]
    q2, q1, q0 = c * d - b * e, 2.0 * (c - a * e), b - a * d
    if abs(q2) < 1e-300:
        roots = [-q0 / q1]
    else:
        disc = q1 * q1 - 4.0 * q2 * q0
        if disc < 0.0:
            raise ValueError("no stationary point")
        sq = math.sqrt(disc)
        roots = [(-q1 + sq) / (2.0 * q2), (-q1 - sq) / (2.0 * q2)]
    best = min(roots, key=lambda t: energy(h, t))
    return best, energy(h, best)
