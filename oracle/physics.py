"""Physical quantities of a fixed wave function (the measurement mode of
Sec. 2.2.3, NVMCCalMode = 1): equal-time pair correlations estimated by
Eq. MC, and the structure factors of Sec. 2.4.2 built from them.

Test infrastructure, like the rest of ``oracle``: tests, the smoke check and
the CPU-baseline leg of the benchmark may call it; the product library never
does.

For a configuration |x> and an operator A, the local estimator of Eq. MC is
    A_loc(x) = <psi|A|x> / <psi|x> = sum_x' <x'|A|x> psi(x') / psi(x)
(real psi): A acts on the ket |x>, each resulting |x'> is weighted by its
amplitude, recomputed from scratch.  <A> is the mean of A_loc over
configurations drawn from rho(x) = |psi(x)|^2 / <psi|psi> (Sec. 3.1.1).

Pair correlations, one Ns x Ns matrix per kind (kind index, operator at
site pair (i, j)):
    0  c^dag_{i up} c_{j up}
    1  c^dag_{i dn} c_{j dn}
    2  n_i n_j,                 n_i = n_{i up} + n_{i dn}
    3  S^z_i S^z_j,             S^z_i = (n_{i up} - n_{i dn}) / 2
    4  S^+_i S^-_j,             S^+_i = c^dag_{i up} c_{i dn}, S^-_i its adjoint
    5  S_i . S_j = S^z_i S^z_j + (S^+_i S^-_j + S^-_i S^+_j) / 2
The off-diagonal kinds (0, 1, 4 and the transverse part of 5) are applied as
operator strings in the canonical Fock basis with their Jordan-Wigner signs;
the diagonal kinds (2, 3) are read off the occupations.

Structure factors (Sec. 2.4.2): X(k) = (1/N_cell) sum_{i,j} exp(-i k.(R_i - R_j))
<X_i^dag X_j>; from the kinds above, n_sigma(k) from 0 / 1, N(k) from 2,
S^z(k) from 3, S(k) from 5.  The quantities of the comparison with exact
diagonalisation (Sec. 4.1.1, Sec. 4.2): the doublon density
D = (1/Ns) sum_i <n_i,up n_i,dn>, the nearest-neighbour spin correlation
S_nn (read as the mean of <S_i . S_j> over nearest-neighbour bonds: the
printed (1/(4 Ns)) sum_{i, mu} on the square lattice, and what reproduces
the printed exact value of the Kondo chain) and S~(k) = S(k) / (3 N_cell).
"""
import math

import numpy as np

from .fock import apply_string
from .hamiltonian import _apply_string_vec, basis

KINDS = ("cdag_c_up", "cdag_c_dn", "n_n", "sz_sz", "sp_sm", "s_s")


def _strings(Ns, i, j):
    """Operator strings (left to right as written) of kinds 0, 1, 4 and of
    S^-_i S^+_j, for the pair (i, j)."""
    up_i, up_j, dn_i, dn_j = i, j, Ns + i, Ns + j
    return {
        0: [("+", up_i), ("-", up_j)],
        1: [("+", dn_i), ("-", dn_j)],
        4: [("+", up_i), ("-", dn_i), ("+", dn_j), ("-", up_j)],
        "sm_sp": [("+", dn_i), ("-", up_i), ("+", up_j), ("-", dn_j)],
    }


class _Local:
    """Local estimators of one configuration n, with the amplitudes of the
    configurations reached from it cached."""

    def __init__(self, wf, n):
        self.wf, self.n, self.Ns = wf, n, wf.Ns
        self.s0, self.l0 = wf.amplitude_slog(n)
        if self.s0 == 0.0:
            raise ZeroDivisionError("psi(x) = 0")
        self.cache = {}
        Ns = wf.Ns
        self.up = np.array([(n >> i) & 1 for i in range(Ns)], np.float64)
        self.dn = np.array([(n >> (Ns + i)) & 1 for i in range(Ns)], np.float64)

    def ratio(self, n2):
        if n2 == self.n:
            return 1.0
        if n2 not in self.cache:
            s1, l1 = self.wf.amplitude_slog(n2)
            self.cache[n2] = 0.0 if s1 == 0.0 else s1 * self.s0 * math.exp(l1 - self.l0)
        return self.cache[n2]

    def loc(self, ops):
        r = apply_string(ops, (1.0, self.n))
        return 0.0 if r is None else r[0] * self.ratio(r[1])

    def entry(self, kind, i, j):
        up, dn = self.up, self.dn
        if kind == 2:
            return (up[i] + dn[i]) * (up[j] + dn[j])
        szsz = 0.25 * (up[i] - dn[i]) * (up[j] - dn[j])
        if kind == 3:
            return szsz
        st = _strings(self.Ns, i, j)
        if kind in (0, 1, 4):
            return self.loc(st[kind])
        return szsz + 0.5 * (self.loc(st[4]) + self.loc(st["sm_sp"]))


def local_correlation(wf, n, kind, i, j):
    """One entry A_loc(x) of local_correlations (for large lattices)."""
    return _Local(wf, n).entry(kind, i, j)


def local_correlations(wf, n):
    """[6, Ns, Ns] array of A_loc(x) for every kind and site pair (Eq. MC)."""
    L = _Local(wf, n)
    Ns = wf.Ns
    out = np.zeros((6, Ns, Ns))
    for kind in range(6):
        for i in range(Ns):
            for j in range(Ns):
                out[kind, i, j] = L.entry(kind, i, j)
    return out


def mean_correlations(wf, configs):
    """Mean of local_correlations over configurations (bitmasks) drawn from
    rho(x): the estimate of Eq. MC."""
    acc = None
    for n in configs:
        v = local_correlations(wf, n)
        acc = v if acc is None else acc + v
    return acc / len(configs)


def exact_correlations(wf):
    """<psi|A|psi>/<psi|psi> for every kind and pair by enumeration of all
    S^z = 0 configurations, weighted by rho(x) (tiny systems only)."""
    N = wf.Ne // 2
    states = basis(wf.Ns, N, N, wf.local_spin, wf.local_sites)
    amps = np.array([wf.amplitude(n) for n in states])
    w = amps ** 2
    keep = np.nonzero(w > 0)[0]
    w = w[keep] / w[keep].sum()
    acc = np.zeros((6, wf.Ns, wf.Ns))
    for k, wk in zip(keep, w):
        acc += wk * local_correlations(wf, states[k])
    return acc


def doublon_density(corr):
    """D = (1/Ns) sum_i <n_i,up n_i,dn>, from n_i^2 = n_i + 2 n_i,up n_i,dn
    and n_i = <c^dag_{i up} c_{i up}> + <c^dag_{i dn} c_{i dn}>."""
    Ns = corr.shape[-1]
    d = np.diagonal(corr[2]) - np.diagonal(corr[0]) - np.diagonal(corr[1])
    return float(0.5 * d.sum() / Ns)


def nn_spin_correlation(ss, bond_i, bond_j):
    """S_nn: the mean over the nearest-neighbour bonds (each undirected bond
    listed once) of (<S_i . S_j> + <S_j . S_i>) / 2; ss is the [Ns, Ns]
    matrix of <S_a . S_b> (kind 5)."""
    tot = sum(0.5 * (ss[i, j] + ss[j, i]) for i, j in zip(bond_i, bond_j))
    return float(tot / len(bond_i))


def state_spin_matrix(Ns, states, vec):
    """[Ns, Ns] matrix of <v| S_a . S_b |v> for a normalised state vector v
    over the basis `states` (any order; exact diagonalisation checks):
    S^z_a S^z_b from the occupations, (S^+_a S^-_b + S^-_a S^+_b)/2 by
    applying the operator strings to every basis state; S_a . S_a =
    3/4 (n_a - 2 n_a,up n_a,dn)."""
    st = np.asarray(states, np.int64)
    order = np.argsort(st)
    sst = st[order]
    p = np.abs(vec) ** 2
    up = np.stack([(st >> i) & 1 for i in range(Ns)], axis=1).astype(np.float64)
    dn = np.stack([(st >> (Ns + i)) & 1 for i in range(Ns)], axis=1).astype(np.float64)
    sz = 0.5 * (up - dn)
    ss = (sz * p[:, None]).T @ sz
    single = p @ (up + dn - 2 * up * dn)

    def overlap(ops):
        new, sign, ok = _apply_string_vec(ops, st)
        k = np.searchsorted(sst, new[ok])
        kc = np.minimum(k, len(sst) - 1)
        hit = sst[kc] == new[ok]
        return float(np.sum(vec[order[kc[hit]]] * sign[ok][hit] * vec[ok][hit]))

    for a in range(Ns):
        ss[a, a] = 0.75 * single[a]
        for b in range(a + 1, Ns):
            t = 0.5 * (overlap([("+", a), ("-", Ns + a), ("+", Ns + b), ("-", b)]) +
                       overlap([("+", Ns + a), ("-", a), ("+", b), ("-", Ns + b)]))
            ss[a, b] += t
            ss[b, a] += t
    return ss


def structure_factor(mat, R, k, n_cell=None):
    """(1/N_cell) sum_{i,j} exp(-i k.(R_i - R_j)) mat[i, j] for one k
    (real part; R: [Ns, d] site positions, k: [d])."""
    Ns = mat.shape[0]
    n_cell = Ns if n_cell is None else n_cell
    ph = np.exp(-1j * (np.asarray(R, np.float64) @ np.asarray(k, np.float64)))
    return float(np.real(ph @ mat @ np.conj(ph)) / n_cell)
