"""Hamiltonian action in the canonical Fock basis and the local energy.

H = H_T + H_U + H_V + J sum S_i.S_j (Sec. 2.3: Eq. GHam, the Hubbard and
Spin models):

* hopping term (i, j, t): -t c^dag_{i s} c_{j s} for both spins s;
* on-site U_i n_i,up n_i,dn and off-site V n_i n_j (diagonal);
* Heisenberg bond (i, j, J): J [S^z_i S^z_j + (S^+_i S^-_j + S^-_i S^+_j)/2]
  with S^+_i = c^dag_{i up} c_{i dn}, S^z_i = (n_i,up - n_i,dn)/2.

The local energy is the estimator of Eq. MC for A = H:
E_loc(x) = sum_x' <x|H|x'> psi(x') / psi(x), each psi(x') recomputed from
scratch (no fast update), with the Jordan-Wigner signs of the Fock basis.
"""
from collections import defaultdict
from itertools import combinations

import numpy as np

from .fock import apply_string


def apply_H(prob, n):
    """H|n> as a dict {n': coefficient}."""
    Ns = prob.lat.Ns
    out = defaultdict(float)
    diag = 0.0
    for i in range(Ns):
        nu = (n >> i) & 1
        nd = (n >> (Ns + i)) & 1
        diag += prob.U[i] * nu * nd
    for i, j, v in zip(prob.V_i, prob.V_j, prob.V_val):
        ni = ((n >> i) & 1) + ((n >> (Ns + i)) & 1)
        nj = ((n >> j) & 1) + ((n >> (Ns + j)) & 1)
        diag += v * ni * nj
    for i, j, t in zip(prob.hop_i, prob.hop_j, prob.hop_t):
        for s in (0, 1):
            r = apply_string([("+", int(i) + Ns * s), ("-", int(j) + Ns * s)], (-float(t), n))
            if r is not None:
                out[r[1]] += r[0]
    for i, j, J in zip(prob.ex_i, prob.ex_j, prob.ex_J):
        i, j, J = int(i), int(j), float(J)
        szi = 0.5 * (((n >> i) & 1) - ((n >> (Ns + i)) & 1))
        szj = 0.5 * (((n >> j) & 1) - ((n >> (Ns + j)) & 1))
        diag += J * szi * szj
        for ops in ([("+", i), ("-", Ns + i), ("+", Ns + j), ("-", j)],
                    [("+", Ns + i), ("-", i), ("+", j), ("-", Ns + j)]):
            r = apply_string(ops, (0.5 * J, n))
            if r is not None:
                out[r[1]] += r[0]
    if diag != 0.0:
        out[n] += diag
    return dict(out)


def local_energy(wf, n):
    """E_loc(x) = sum_x' <x|H|x'> psi(x')/psi(x) (real symmetric H)."""
    s0, l0 = wf.amplitude_slog(n)
    if s0 == 0.0:
        raise ZeroDivisionError("psi(x) = 0")
    e = 0.0
    for n2, coef in apply_H(wf.prob, n).items():
        if n2 == n:
            e += coef
            continue
        s1, l1 = wf.amplitude_slog(n2)
        if s1 != 0.0:
            e += coef * s1 * s0 * np.exp(l1 - l0)
    return float(e)


def basis(Ns, N_up, N_dn, local_spin=False, local_sites=None):
    """All S^z-fixed configurations as bitmasks (no doublons if local_spin;
    exactly one electron on each site of the local_sites mask)."""
    if local_sites is not None:
        return _basis_local_sites(Ns, N_up, N_dn, np.asarray(local_sites, bool))
    out = []
    for ups in combinations(range(Ns), N_up):
        mu = sum(1 << i for i in ups)
        if local_spin and N_up + N_dn == Ns:
            out.append(mu | sum(1 << (Ns + i) for i in range(Ns) if i not in ups))
            continue
        for dns in combinations(range(Ns), N_dn):
            if local_spin and set(ups) & set(dns):
                continue
            out.append(mu | sum(1 << (Ns + i) for i in dns))
    return out


def _basis_local_sites(Ns, N_up, N_dn, mask):
    loc = [i for i in range(Ns) if mask[i]]
    itin = [i for i in range(Ns) if not mask[i]]
    out = []
    for k in range(len(loc) + 1):            # up spins among the local sites
        cu, cd = N_up - k, N_dn - (len(loc) - k)
        if not (0 <= cu <= len(itin) and 0 <= cd <= len(itin)):
            continue
        for lu in combinations(loc, k):
            up_loc = set(lu)
            base = sum(1 << i for i in lu) | sum(1 << (Ns + i) for i in loc if i not in up_loc)
            for ups in combinations(itin, cu):
                m1 = base | sum(1 << i for i in ups)
                for dns in combinations(itin, cd):
                    out.append(m1 | sum(1 << (Ns + i) for i in dns))
    return out


def hamiltonian_matrix(prob, states):
    """Sparse H in the given basis (scipy CSR)."""
    import scipy.sparse as sp
    index = {s: k for k, s in enumerate(states)}
    rows, cols, vals = [], [], []
    for k, s in enumerate(states):
        for s2, coef in apply_H(prob, s).items():
            if s2 in index:
                rows.append(index[s2])
                cols.append(k)
                vals.append(coef)
    n = len(states)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def _apply_string_vec(ops, n):
    """Vectorised apply_string over an int64 array of bitmasks: returns
    (new states, Jordan-Wigner signs, validity mask)."""
    n = n.copy()
    valid = np.ones(n.shape, bool)
    sign = np.ones(n.shape)
    for kind, I in reversed(ops):
        bit = (n >> I) & 1
        valid &= (bit == 1) if kind == "-" else (bit == 0)
        below = np.bitwise_count(n & ((1 << I) - 1)) & 1
        sign *= np.where(below == 1, -1.0, 1.0)
        n ^= (1 << I)
    return n, sign, valid


def hamiltonian_matrix_vec(prob, states):
    """The matrix of apply_H, built term by term over all states at once
    (same operator strings and signs; used where the basis is large)."""
    import scipy.sparse as sp
    Ns = prob.lat.Ns
    st = np.asarray(states, np.int64)
    order = np.argsort(st)
    sst = st[order]
    nS = st.size
    rows, cols, vals = [], [], []
    idx = np.arange(nS)

    def add(new, coef, ok):
        k = np.searchsorted(sst, new[ok])
        hit = (k < nS) & (sst[np.minimum(k, nS - 1)] == new[ok])
        rows.append(order[np.minimum(k, nS - 1)][hit])
        cols.append(idx[ok][hit])
        vals.append(coef[ok][hit])

    up = [(st >> i) & 1 for i in range(Ns)]
    dn = [(st >> (Ns + i)) & 1 for i in range(Ns)]
    diag = np.zeros(nS)
    for i in range(Ns):
        diag += prob.U[i] * up[i] * dn[i]
    for i, j, v in zip(prob.V_i, prob.V_j, prob.V_val):
        diag += v * (up[i] + dn[i]) * (up[j] + dn[j])
    for i, j, t in zip(prob.hop_i, prob.hop_j, prob.hop_t):
        for s in (0, 1):
            new, sg, ok = _apply_string_vec([("+", int(i) + Ns * s), ("-", int(j) + Ns * s)], st)
            add(new, -float(t) * sg, ok)
    for i, j, J in zip(prob.ex_i, prob.ex_j, prob.ex_J):
        i, j, J = int(i), int(j), float(J)
        diag += J * 0.25 * (up[i] - dn[i]) * (up[j] - dn[j])
        for ops in ([("+", i), ("-", Ns + i), ("+", Ns + j), ("-", j)],
                    [("+", Ns + i), ("-", i), ("+", j), ("-", Ns + j)]):
            new, sg, ok = _apply_string_vec(ops, st)
            add(new, 0.5 * J * sg, ok)
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nS, nS))


def ground_state_energy(prob, two_sz=0):
    """Exact diagonalisation in the sector 2 S^z = two_sz (dense below 3000
    states, else Lanczos via scipy eigsh)."""
    states = basis(prob.lat.Ns, (prob.Ne + two_sz) // 2, (prob.Ne - two_sz) // 2,
                   prob.local_spin, getattr(prob, "local_sites", None))
    H = hamiltonian_matrix_vec(prob, states)
    if len(states) <= 3000:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    from scipy.sparse.linalg import eigsh
    return float(eigsh(H, k=1, which="SA", tol=1e-12)[0][0])
