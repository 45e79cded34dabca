"""Test helpers: oracle-side evaluation of labelled configurations, and the
GPU context factory (tests only)."""
import math
import os

import numpy as np

from oracle import fock
from oracle.hamiltonian import local_energy
from oracle.wavefunction import Wavefunction


def labelled_slog(wf, ele):
    """(sign, log|psi|) of the labelled configuration prod c+_{r_n up} prod c+_{r_m dn}|0>."""
    n = fock.from_labels(ele, wf.Ns)
    s, l = wf.amplitude_slog(n)
    return s * fock.label_sign(ele, wf.Ns), l


def apply_move(ele, move, N):
    kind, a, b = move
    e = list(int(x) for x in ele)
    if kind == 0:
        e[a] = b
    else:
        e[a], e[b] = e[b], e[a]
    return e


def move_valid(ele, move, N, Ns, local_spin):
    kind, a, b = move
    up = {int(s) for s in ele[:N]}
    dn = {int(s) for s in ele[N:]}
    if kind == 0:
        same = up if a < N else dn
        other = dn if a < N else up
        if b in same:
            return False
        if local_spin and b in other:
            return False
        return True
    i, j = int(ele[a]), int(ele[b])
    return i != j and i not in dn and j not in up


def oracle_ratio(wf, ele, move):
    s0, l0 = labelled_slog(wf, ele)
    e2 = apply_move(ele, move, len(ele) // 2)
    s1, l1 = labelled_slog(wf, e2)
    if s1 == 0.0:
        return 0.0
    return s1 * s0 * math.exp(l1 - l0)


def oracle_measure(wf, ele):
    n = fock.from_labels(ele, wf.Ns)
    return local_energy(wf, n), wf.log_derivatives(n)


def condition_ok(wf, ele, limit=1e8):
    X, _ = wf.X(fock.from_labels(ele, wf.Ns))
    return np.linalg.cond(X) < limit


def random_moves(rng, ele, N, Ns, local_spin, k, p_ex=0.5):
    Ne = 2 * N
    out = []
    while len(out) < k:
        if local_spin or rng.random() < p_ex:
            mv = (1, int(rng.integers(N)), int(N + rng.integers(N)))
        else:
            mv = (0, int(rng.integers(Ne)), int(rng.integers(Ns)))
        if move_valid(ele, mv, N, Ns, local_spin):
            out.append(mv)
    return out
