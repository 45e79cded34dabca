"""Pfaffians of real skew-symmetric matrices (Sec. 3.2.1: <x|phi_Pf> is
(Ne/2)! Pf(X); Pf(X)^2 = det X).

``pfaffian`` is Parlett-Reid elimination: congruence transforms by unit
lower-triangular matrices (which leave the Pfaffian unchanged, by
Pf(B A B^T) = det(B) Pf(A), Appendix C) reduce A column pair by column pair;
the Pfaffian is then the product of the (2k, 2k+1) pivots, with a sign flip
for every symmetric row/column interchange.  Written from the method's
description, not from PFAPACK.

``pfaffian_expand`` is the definition itself (expansion along the first
row), exponential cost, for pins on tiny matrices.
"""
import math

import numpy as np


def pfaffian_slog(A):
    """Return (sign, log|Pf(A)|) of a real skew-symmetric matrix A
    (sign 0 and -inf when Pf(A) = 0)."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    if n % 2 == 1:
        return 0.0, -math.inf
    sign = 1.0
    logabs = 0.0
    for k in range(0, n - 1, 2):
        # Pivot: largest entry of column k below the diagonal block.
        p = k + 1 + int(np.argmax(np.abs(A[k + 1:, k])))
        if p != k + 1:
            A[[k + 1, p], :] = A[[p, k + 1], :]
            A[:, [k + 1, p]] = A[:, [p, k + 1]]
            sign = -sign
        piv = A[k, k + 1]
        if piv == 0.0:
            return 0.0, -math.inf
        if piv < 0:
            sign = -sign
        logabs += math.log(abs(piv))
        if k + 2 < n:
            # Column/row op: col_i -= tau_i col_{k+1}, row_i -= tau_i row_{k+1}
            # with tau_i = A[k, i] / A[k, k+1] zeroes A[k, k+2:].
            tau = A[k, k + 2:] / piv
            # Trailing block update A[i,j] += -tau_i A[k+1,j] + tau_j A[k+1,i].
            r = A[k + 1, k + 2:].copy()
            A[k + 2:, k + 2:] += np.outer(r, tau) - np.outer(tau, r)
            A[k, k + 2:] = 0.0
            A[k + 2:, k] = 0.0
    return sign, logabs


def pfaffian(A):
    s, l = pfaffian_slog(A)
    return s * math.exp(l) if s != 0.0 else 0.0


def pfaffian_expand(A):
    """Pf(A) = sum_{j>0} (-1)^{j+1} A[0, j] Pf(A without rows/cols 0, j)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n == 0:
        return 1.0
    if n % 2 == 1:
        return 0.0
    total = 0.0
    for j in range(1, n):
        if A[0, j] == 0.0:
            continue
        keep = [k for k in range(1, n) if k != j]
        total += (-1) ** (j + 1) * A[0, j] * pfaffian_expand(A[np.ix_(keep, keep)])
    return total
