"""Canonical Fock basis over spin-orbitals I = i + Ns*sigma (Sec. 3.2.1).

A basis state is a Python int bitmask n; bit I set means orbital I is
occupied.  The state is c^dag_{I_1} c^dag_{I_2} ... c^dag_{I_K} |0> with
I_1 < I_2 < ... < I_K (the real-space configuration |x> of Sec. 3.1.1 with
the electrons in ascending orbital order).  Creation and annihilation carry
the Jordan-Wigner sign (-1)^(number of occupied orbitals below I).
"""


def popcount(n: int) -> int:
    return bin(n).count("1")


def cdag(I: int, state):
    """Apply c^dag_I to (coef, n); return None if the result vanishes."""
    if state is None:
        return None
    coef, n = state
    if n >> I & 1:
        return None
    sign = -1.0 if popcount(n & ((1 << I) - 1)) & 1 else 1.0
    return coef * sign, n | (1 << I)


def c(I: int, state):
    if state is None:
        return None
    coef, n = state
    if not (n >> I & 1):
        return None
    sign = -1.0 if popcount(n & ((1 << I) - 1)) & 1 else 1.0
    return coef * sign, n & ~(1 << I)


def apply_string(ops, state):
    """Apply an operator string, rightmost first.  ops: list of
    ('+', I) or ('-', I) written left to right as in the formula."""
    for kind, I in reversed(ops):
        state = cdag(I, state) if kind == "+" else c(I, state)
        if state is None:
            return None
    return state


def occupied(n: int, norb: int):
    return [I for I in range(norb) if n >> I & 1]


def from_labels(ele, Ns: int) -> int:
    """Bitmask of a labelled configuration (ele[n] for n < N up, else down)."""
    N = len(ele) // 2
    n = 0
    for k, site in enumerate(ele):
        I = int(site) + (Ns if k >= N else 0)
        n |= 1 << I
    return n


def label_sign(ele, Ns: int) -> float:
    """Sign of the permutation taking the labelled product
    prod_n c^dag_{r_n up} prod_m c^dag_{r_m dn} |0> to the ascending order:
    |x_labelled> = label_sign * |x_canonical>."""
    N = len(ele) // 2
    orbs = [int(s) + (Ns if k >= N else 0) for k, s in enumerate(ele)]
    inv = 0
    for a in range(len(orbs)):
        for b in range(a + 1, len(orbs)):
            if orbs[a] > orbs[b]:
                inv += 1
    return -1.0 if inv & 1 else 1.0
