"""Quantum-number projection of the pair-product part (Sec. 3.2.2, Eqs. momP
and pointP): psi(x) = P(x) <x| L |phi_Pf> (the wave function of Sec. 3.2,
correlation factors P applied after the projector), with

    L_K = (1/Ns) sum_R exp(i K.R) T_R,   L_P = (1/N_g) sum_p g(p)^-1 T_p,

T_g c^dag_{r s} T_g^-1 = s_g(r) c^dag_{g(r) s}: a site map with the sign
that an anti-periodic boundary gives a fermion carried across it (App. A).

Test infrastructure, like the rest of ``oracle``.

<x| T_g |phi> = <T_g^-1 x | phi>: the configuration's creation operators
are mapped by the inverse operation (with its boundary signs) and put back
in canonical order by the operator algebra of ``fock``; the Pfaffian of the
mapped configuration follows.  The weights may be complex for the checks of
the projector itself; ProjectedWavefunction (energies, sampling) needs real
ones (momenta with components 0 or pi, real characters).
"""
import cmath
import math

import numpy as np

from .fock import apply_string, occupied


class SymOp:
    """A lattice symmetry: site r -> perm[r] with fermion sign sign[r]."""

    def __init__(self, perm, sign, label=""):
        self.perm = np.asarray(perm, np.int64)
        self.sign = np.asarray(sign, np.float64)
        self.label = label
        inv = np.empty_like(self.perm)
        inv[self.perm] = np.arange(self.perm.size)
        self.inv = inv
        # T_g^-1 c^dag_q T_g = sign[g^-1(q)] c^dag_{g^-1(q)}
        self.inv_sign = self.sign[inv]

    def compose(self, other):
        """self after other: r -> self(other(r)), signs multiplied."""
        return SymOp(self.perm[other.perm], other.sign * self.sign[other.perm],
                     f"{self.label}*{other.label}")


def translations(lat):
    """T_R for every R = (dx, dy) of the lattice (Lattice.site folds the
    image into the cell and returns its boundary sign)."""
    ops = []
    for dy in range(lat.Ly):
        for dx in range(lat.Lx):
            perm, sign = [], []
            for i in range(lat.Ns):
                x, y = lat.xy(i)
                j, s = lat.site(x + dx, y + dy)
                perm.append(j)
                sign.append(s)
            ops.append((SymOp(perm, sign, f"T({dx},{dy})"), (dx, dy)))
    return ops


def point_ops(lat):
    """The point operations of the square lattice about site 0 that map the
    lattice onto itself: identity, the rotations by 90, 180 and 270 degrees
    (Lx = Ly only), and the reflections x -> -x, y -> -y and their
    diagonal partners (Lx = Ly only).  Returned as (SymOp, name)."""
    maps = [("E", lambda x, y: (x, y)), ("C2", lambda x, y: (-x, -y)),
            ("Mx", lambda x, y: (-x, y)), ("My", lambda x, y: (x, -y))]
    if lat.Lx == lat.Ly:
        maps += [("C4", lambda x, y: (-y, x)), ("C4^3", lambda x, y: (y, -x)),
                 ("Md", lambda x, y: (y, x)), ("Md'", lambda x, y: (-y, -x))]
    ops = []
    for name, f in maps:
        perm, sign = [], []
        for i in range(lat.Ns):
            x, y = lat.xy(i)
            j, s = lat.site(*f(x, y))
            perm.append(j)
            sign.append(s)
        ops.append((SymOp(perm, sign, name), name))
    return ops


def momentum_weights(trans, K):
    """Eq. momP: w_R = exp(i K.R) / Ns for the translations returned by
    translations()."""
    n = len(trans)
    return [(op, cmath.exp(1j * (K[0] * R[0] + K[1] * R[1])) / n) for op, R in trans]


def combine(a, b):
    """L_a L_b as one weighted operation list (every pair composed)."""
    return [(oa.compose(ob), wa * wb) for oa, wa in a for ob, wb in b]


def mapped_configuration(op, n, Ns):
    """T_g^-1 |x> = sign |x'> in the canonical basis: returns (sign, x')."""
    orbs = occupied(n, 2 * Ns)
    string = []
    sgn = 1.0
    for I in orbs:                       # canonical product, ascending I
        s, site = (1, I - Ns) if I >= Ns else (0, I)
        q = int(op.inv[site])
        sgn *= op.inv_sign[site]
        string.append(("+", q + Ns * s))
    r = apply_string(string, (sgn, 0))
    return r


def pair_amplitude_slog(wf, n):
    """(sign, log|<x|phi_Pf>|) including (Ne/2)!, without correlation factors."""
    from .pfaffian import pfaffian_slog
    X, _ = wf.X(n)
    s, l = pfaffian_slog(X)
    if s == 0.0:
        return 0.0, -math.inf
    return s, l + math.lgamma(wf.Ne // 2 + 1)


def projected_pair_amplitude(wf, n, weighted_ops):
    """<x| L |phi_Pf> = sum_g w_g <T_g^-1 x|phi_Pf> (complex if the weights are)."""
    tot = 0.0
    for op, w in weighted_ops:
        r = mapped_configuration(op, n, wf.Ns)
        if r is None:
            continue
        sgn, n2 = r
        s, l = pair_amplitude_slog(wf, n2)
        if s != 0.0:
            tot = tot + w * sgn * s * math.exp(l)
    return tot


class ProjectedWavefunction:
    """psi(x) = P(x) <x| L |phi_Pf> for real weights: the same interface as
    Wavefunction for amplitudes, local energies and O_k."""

    def __init__(self, wf, weighted_ops):
        for _, w in weighted_ops:
            if abs(complex(w).imag) > 1e-14:
                raise ValueError("ProjectedWavefunction needs real weights")
        self.base = wf
        self.ops = [(op, float(complex(w).real)) for op, w in weighted_ops]
        self.prob, self.Ns, self.Ne = wf.prob, wf.Ns, wf.Ne
        self.local_spin, self.local_sites = wf.local_spin, wf.local_sites
        self.params = wf.params

    def amplitude_slog(self, n):
        up, dn = self.base.occ(n)
        if self.local_spin and np.any(up * dn):
            return 0.0, -math.inf
        if self.local_sites is not None and np.any((up + dn)[self.local_sites] != 1):
            return 0.0, -math.inf
        a = projected_pair_amplitude(self.base, n, self.ops)
        if a == 0.0:
            return 0.0, -math.inf
        return (1.0 if a > 0 else -1.0), (math.log(abs(a)) + self.base.log_correlation(n)
                                          + self.base.mlp_log(n))

    def amplitude(self, n):
        s, l = self.amplitude_slog(n)
        return s * math.exp(l) if s != 0.0 else 0.0

    def log_derivatives(self, n):
        """O_k = d ln psi / d alpha_k (Sec. 3.3.1) of the projected state.
        The correlation factors multiply the projected pair product, so their
        O_k are those of x itself.  The pair-orbital part is the derivative of
        ln sum_g w_g <T_g^-1 x|phi>: each term contributes its own
        d ln Pf / d f (Eq. DiffPf, on the mapped configuration) weighted by
        its share of the sum."""
        base = self.base
        out = base.log_derivatives(n)
        k0, k1 = base.n_g + base.n_v, base.n_g + base.n_v + base.n_f
        num = np.zeros(k1 - k0)
        den = 0.0
        for op, w in self.ops:
            r = mapped_configuration(op, n, self.Ns)
            if r is None:
                continue
            sgn, n2 = r
            s, l = pair_amplitude_slog(base, n2)
            if s == 0.0:
                continue
            a = w * sgn * s * math.exp(l)
            num += a * base.log_derivatives(n2)[k0:k1]
            den += a
        out[k0:k1] = num / den
        return out
