"""Seeded synthetic inputs: lattices, Hamiltonian term lists, variational
layouts, initial parameters and initial electron configurations.

This module builds problem instances only.  It holds none of the sampling,
Pfaffian, local-energy, derivative or SR arithmetic: both the CUDA path and
the CPU oracle receive the arrays it returns.

Conventions (they follow the paper's Standard-mode models):

* Sites ``i = x + Lx*y``; spin-orbital ``I = i + Ns*sigma`` (sigma = 0 up,
  1 down), as in the definition of the Pfaffian wave function (Sec. 3.2.1).
* Hopping terms are directed: a term ``(i, j, t)`` stands for
  ``-t c^dag_{i sigma} c_{j sigma}`` for both spins (the Hubbard model of
  Sec. 2.3); every bond is listed in both directions with the same real t.
  Anti-periodic boundaries multiply t across the cell boundary by -1
  (Appendix A, phase = pi).
* Heisenberg bonds ``(i, j, J)`` stand for ``J S_i . S_j``, each bond once.
* Variational parameters are one real vector laid out as
  ``[g (n_g) | v (n_v) | f (n_f)]``: Gutzwiller classes, Jastrow classes and
  pair-orbital classes.  ``f_ij = f_sign[i,j] * p_f[f_idx[i,j]]`` (zero where
  ``f_idx = -1``); the sign carries the anti-periodic translation sign of
  Appendix A.
* Electron labels: ``ele[n]`` for ``n < N`` is the site of up electron n,
  ``ele[N+m]`` the site of down electron m (N = Ne/2, S^z = 0).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


# ---------------------------------------------------------------------------
# Lattices
# ---------------------------------------------------------------------------
@dataclass
class Lattice:
    Lx: int
    Ly: int
    bc_x: int = 1   # +1 periodic, -1 anti-periodic
    bc_y: int = 1

    @property
    def Ns(self) -> int:
        return self.Lx * self.Ly

    def site(self, x: int, y: int) -> tuple[int, int]:
        """Fold (x, y) into the cell; return (site index, boundary sign)."""
        s = 1
        while x < 0:
            x += self.Lx
            s *= self.bc_x
        while x >= self.Lx:
            x -= self.Lx
            s *= self.bc_x
        while y < 0:
            y += self.Ly
            s *= self.bc_y
        while y >= self.Ly:
            y -= self.Ly
            s *= self.bc_y
        return x + self.Lx * y, s

    def xy(self, i: int) -> tuple[int, int]:
        return i % self.Lx, i // self.Lx


def chain(L: int, bc: int = 1) -> Lattice:
    return Lattice(L, 1, bc, 1)


def square(Lx: int, Ly: int, bc_x: int = 1, bc_y: int = 1) -> Lattice:
    return Lattice(Lx, Ly, bc_x, bc_y)


def translation_ops(lat: Lattice):
    """Every lattice translation R = (dx, dy) as a site map with boundary
    signs (App. A): perm[g, i] = the site of i + R folded into the cell,
    sign[g, i] = the sign its folding picks up; g = dx + Lx dy.  Geometry
    only: the operations of vmc_set_projection's momentum projection."""
    G = lat.Ns
    perm = np.zeros((G, lat.Ns), np.int32)
    sign = np.ones((G, lat.Ns), np.int8)
    for dy in range(lat.Ly):
        for dx in range(lat.Lx):
            g = dx + lat.Lx * dy
            for i in range(lat.Ns):
                x, y = lat.xy(i)
                perm[g, i], sign[g, i] = lat.site(x + dx, y + dy)
    return perm, sign


def _neighbour_vectors(lat: Lattice, order: int):
    """Displacements of nearest (order 1) or next-nearest (order 2) bonds,
    one per undirected bond direction."""
    if lat.Ly == 1:
        return [(1, 0)] if order == 1 else [(2, 0)]
    if order == 1:
        return [(1, 0), (0, 1)]
    return [(1, 1), (1, -1)]


def bonds(lat: Lattice, order: int = 1):
    """Undirected bonds (i, j, boundary sign), each bond once."""
    out = []
    for i in range(lat.Ns):
        x, y = lat.xy(i)
        for dx, dy in _neighbour_vectors(lat, order):
            j, s = lat.site(x + dx, y + dy)
            if j == i:
                continue
            out.append((i, j, s))
    return out


def hopping_terms(lat: Lattice, t: float = 1.0, t2: float = 0.0):
    """Directed hopping terms (both directions) for -t sum c^dag_i c_j."""
    hi, hj, ht = [], [], []
    for order, amp in ((1, t), (2, t2)):
        if amp == 0.0:
            continue
        for i, j, s in bonds(lat, order):
            hi += [i, j]
            hj += [j, i]
            ht += [amp * s, amp * s]
    return (np.asarray(hi, np.int32), np.asarray(hj, np.int32),
            np.asarray(ht, np.float64))


def heisenberg_bonds(lat: Lattice, J1: float = 1.0, J2: float = 0.0):
    bi, bj, bJ = [], [], []
    for order, amp in ((1, J1), (2, J2)):
        if amp == 0.0:
            continue
        for i, j, _ in bonds(lat, order):
            bi.append(i)
            bj.append(j)
            bJ.append(amp)
    return (np.asarray(bi, np.int32), np.asarray(bj, np.int32),
            np.asarray(bJ, np.float64))


# ---------------------------------------------------------------------------
# Variational layouts
# ---------------------------------------------------------------------------
def sublattice_f_layout(lat: Lattice, Wsub: int, Lsub: int):
    """Pair-orbital classes under the Wsub x Lsub sublattice structure of
    Sec. 3.2.1 (sublattice paragraph) with the boundary signs of Appendix A.

    The pair (i, j) is translated by the lattice vector that brings i into
    the sublattice unit cell; j follows and collects the anti-periodic sign.
    Class = (cell position of i) * Ns + (translated j).
    """
    Ns = lat.Ns
    f_idx = np.full((Ns, Ns), -1, np.int32)
    f_sign = np.zeros((Ns, Ns), np.int8)
    used = {}
    for i in range(Ns):
        xi, yi = lat.xy(i)
        rx, ry = -(xi - xi % Wsub), -(yi - yi % Lsub)
        cell = (xi % Wsub) + Wsub * (yi % Lsub)
        for j in range(Ns):
            xj, yj = lat.xy(j)
            jp, s = lat.site(xj + rx, yj + ry)
            key = cell * Ns + jp
            if key not in used:
                used[key] = len(used)
            f_idx[i, j] = used[key]
            f_sign[i, j] = s
    return f_idx.reshape(-1), f_sign.reshape(-1), len(used)


def full_f_layout(Ns: int):
    """One class per (i, j): no symmetry reduction."""
    f_idx = np.arange(Ns * Ns, dtype=np.int32)
    f_sign = np.ones(Ns * Ns, np.int8)
    return f_idx, f_sign, Ns * Ns


def jastrow_chain_layout(lat: Lattice, max_dist: int = 2):
    """Jastrow classes by ring distance 1..max_dist (C1: nearest + next)."""
    Ns = lat.Ns
    v = np.full((Ns, Ns), -1, np.int32)
    for i in range(Ns):
        for j in range(Ns):
            d = abs(i - j)
            d = min(d, Ns - d)
            if 1 <= d <= max_dist:
                v[i, j] = d - 1
    return v.reshape(-1), max_dist


def jastrow_distance_layout(lat: Lattice):
    """One Jastrow class per symmetry-distinct minimum-image displacement
    (a, b) = sorted(|dx|, |dy|), excluding (0, 0)."""
    Ns = lat.Ns
    keys = {}
    for a in range(lat.Lx // 2 + 1):
        for b in range(a, lat.Ly // 2 + 1):
            if (a, b) != (0, 0):
                keys[(a, b)] = len(keys)
    v = np.full((Ns, Ns), -1, np.int32)
    for i in range(Ns):
        xi, yi = lat.xy(i)
        for j in range(Ns):
            if i == j:
                continue
            xj, yj = lat.xy(j)
            dx = abs(xi - xj)
            dx = min(dx, lat.Lx - dx)
            dy = abs(yi - yj)
            dy = min(dy, lat.Ly - dy)
            a, b = sorted((dx, dy))
            v[i, j] = keys[(a, b)]
    return v.reshape(-1), len(keys)


# ---------------------------------------------------------------------------
# Initial parameters: U = 0 pairing (Appendix B) + seeded noise
# ---------------------------------------------------------------------------
def single_particle_matrix(Ns, hop_i, hop_j, hop_t):
    h = np.zeros((Ns, Ns))
    for i, j, t in zip(hop_i, hop_j, hop_t):
        h[i, j] += -t
    return h


def free_fermion_orbitals(lat: Lattice, hop, N: int):
    """Lowest N single-particle orbitals (real).  For a chain whose top shell
    is degenerate, the standing wave cos(k x) is chosen (invariant, up to
    sign, under translation by two sites); for 2D lattices a shell gap is
    required."""
    Ns = lat.Ns
    if lat.Ly == 1:
        L = lat.Lx
        shift = 0.0 if lat.bc_x == 1 else math.pi / L
        orbs = []
        for q in range(L):
            k = 2 * math.pi * q / L + shift
            if k > math.pi + 1e-12:
                k -= 2 * math.pi
            orbs.append((k, q))
        cand = []
        seen = set()
        for k, _ in orbs:
            ka = round(abs(k), 12)
            if ka in seen:
                continue
            seen.add(ka)
            e = -2.0 * math.cos(ka)
            x = np.arange(L)
            if ka == 0.0 or abs(ka - math.pi) < 1e-12:
                vec = np.cos(ka * x)
                cand.append((e, 0, vec / np.linalg.norm(vec)))
            else:
                c = np.cos(ka * x)
                s = np.sin(ka * x)
                cand.append((e, 0, c / np.linalg.norm(c)))
                cand.append((e, 1, s / np.linalg.norm(s)))
        cand.sort(key=lambda z: (round(z[0], 10), z[1]))
        return np.stack([c[2] for c in cand[:N]], axis=1)
    h = single_particle_matrix(Ns, *hop)
    w, V = np.linalg.eigh(h)
    if N < Ns and w[N] - w[N - 1] < 1e-9:
        raise ValueError("open shell at U=0; choose other boundary conditions")
    return V[:, :N]


def project_to_classes(fmat, f_idx, f_sign, n_f):
    """Average f_ij * sign_ij over each class (exact for a symmetric f)."""
    acc = np.zeros(n_f)
    cnt = np.zeros(n_f)
    fi = f_idx.reshape(-1)
    fs = f_sign.reshape(-1).astype(np.float64)
    m = fi >= 0
    np.add.at(acc, fi[m], fmat.reshape(-1)[m] * fs[m])
    np.add.at(cnt, fi[m], 1.0)
    return acc / np.maximum(cnt, 1.0)


def initial_configs(Ns: int, Ne: int, n_walkers: int, local_spin: bool,
                    seed: int, local_sites=None) -> np.ndarray:
    """Random electron placements, int32 [n_walkers, Ne] in label order.
    With a local_sites mask (Kondo local spins) each marked site receives
    exactly one electron, half of them up (rounded down), and the remaining
    electrons go to unmarked sites."""
    rng = np.random.default_rng(seed)
    N = Ne // 2
    out = np.empty((n_walkers, Ne), np.int32)
    if local_sites is not None:
        loc = np.flatnonzero(np.asarray(local_sites, bool))
        itin = np.flatnonzero(~np.asarray(local_sites, bool))
        k = len(loc) // 2
        for w in range(n_walkers):
            lp = rng.permutation(loc)
            out[w, :k] = lp[:k]
            out[w, k:N] = rng.choice(itin, N - k, replace=False)
            out[w, N:N + len(loc) - k] = lp[k:]
            out[w, N + len(loc) - k:] = rng.choice(itin, N - (len(loc) - k), replace=False)
        return out
    for w in range(n_walkers):
        if local_spin:
            p = rng.permutation(Ns)
            out[w, :N] = p[:N]
            out[w, N:] = p[N:Ne]
        else:
            out[w, :N] = rng.choice(Ns, N, replace=False)
            out[w, N:] = rng.choice(Ns, N, replace=False)
    return out


# ---------------------------------------------------------------------------
# Problem container and the workloads
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    lat: Lattice
    Ne: int
    hop_i: np.ndarray
    hop_j: np.ndarray
    hop_t: np.ndarray
    U: np.ndarray
    ex_i: np.ndarray
    ex_j: np.ndarray
    ex_J: np.ndarray
    local_spin: bool
    g_idx: np.ndarray
    n_g: int
    v_idx: np.ndarray
    n_v: int
    f_idx: np.ndarray
    f_sign: np.ndarray
    n_f: int
    params: np.ndarray
    p_exchange: float
    n_hidden: int = 0
    V_i: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    V_j: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    V_val: np.ndarray = field(default_factory=lambda: np.zeros(0))
    meta: dict = field(default_factory=dict)
    # per-site local-spin constraint (exactly one electron on each marked
    # site); None = none, or all sites when local_spin is set
    local_sites: np.ndarray | None = None

    @property
    def Ns(self) -> int:
        return self.lat.Ns

    @property
    def N(self) -> int:
        return self.Ne // 2

    @property
    def n_mlp(self) -> int:
        H, C = self.n_hidden, 2 * self.lat.Ns
        return H * C + 2 * H + 1 if H > 0 else 0

    @property
    def Np(self) -> int:
        return self.n_g + self.n_v + self.n_f + self.n_mlp

    def f_matrix(self, params=None) -> np.ndarray:
        p = self.params if params is None else params
        pf = p[self.n_g + self.n_v:self.n_g + self.n_v + self.n_f]
        fi = self.f_idx.reshape(-1)
        f = np.where(fi >= 0, pf[np.maximum(fi, 0)], 0.0) * self.f_sign.reshape(-1)
        return f.reshape(self.Ns, self.Ns)

    def copy_with(self, **kw) -> "Problem":
        d = dict(self.__dict__)
        d.update(kw)
        return Problem(**d)


def make_problem(name, lat, Ne, *, t=1.0, t2=0.0, U=0.0, J1=0.0, J2=0.0,
                 local_spin=False, sub=(1, 1), f_full=False, jastrow="none",
                 gutzwiller=True, noise=0.05, seed=0, p_exchange=None,
                 f_init="pairing", mlp_hidden=0, mlp_std=0.01):
    Ns = lat.Ns
    N = Ne // 2
    hop = hopping_terms(lat, t, t2) if (t != 0.0 or t2 != 0.0) else (
        np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    ex = heisenberg_bonds(lat, J1, J2) if (J1 != 0.0 or J2 != 0.0) else (
        np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    if f_full:
        f_idx, f_sign, n_f = full_f_layout(Ns)
    else:
        f_idx, f_sign, n_f = sublattice_f_layout(lat, *sub)
    if jastrow == "chain":
        v_idx, n_v = jastrow_chain_layout(lat, 2)
    elif jastrow == "distance":
        v_idx, n_v = jastrow_distance_layout(lat)
    else:
        v_idx, n_v = np.full(Ns * Ns, -1, np.int32), 0
    if gutzwiller and not local_spin:
        g_idx, n_g = np.zeros(Ns, np.int32), 1
    else:
        g_idx, n_g = np.full(Ns, -1, np.int32), 0
    # U = 0 pairing from the orbitals of the hopping matrix; spin models use
    # the nearest-neighbour hopping of the same lattice for this purpose.
    if f_init == "pairing":
        hop_for_f = hop if hop[0].size else hopping_terms(lat, 1.0, 0.0)
        Phi = free_fermion_orbitals(lat, hop_for_f, N)
        fmat = Phi @ Phi.T
        pf = project_to_classes(fmat, f_idx, f_sign, n_f)
        pf = pf / np.max(np.abs(pf))
    else:
        pf = np.zeros(n_f)
    rng = np.random.default_rng(seed)
    if noise:
        pf = pf + rng.uniform(-noise, noise, n_f)
    params = np.concatenate([np.zeros(n_g), np.zeros(n_v), pf])
    if mlp_hidden:
        # MLP correlation factor [W1 (H x 2Ns, row-major) | b1 (H) | w2 (H) | b2],
        # weights and biases N(0, mlp_std^2), seeded after the pair orbitals.
        H, C = int(mlp_hidden), 2 * Ns
        params = np.concatenate([params, rng.normal(0.0, mlp_std, H * C + 2 * H + 1)])
    if p_exchange is None:
        p_exchange = 1.0 if local_spin else (0.5 if U >= 4.0 else 0.0)
    return Problem(name=name, lat=lat, Ne=Ne, hop_i=hop[0], hop_j=hop[1],
                   hop_t=hop[2], U=np.full(Ns, float(U)), ex_i=ex[0],
                   ex_j=ex[1], ex_J=ex[2], local_spin=bool(local_spin),
                   g_idx=g_idx, n_g=n_g, v_idx=v_idx, n_v=n_v, f_idx=f_idx,
                   f_sign=f_sign, n_f=n_f, params=params,
                   p_exchange=float(p_exchange), n_hidden=int(mlp_hidden))


def ring8_hubbard(noise=0.05, seed=0, U=4.0):
    """1D Hubbard ring, 8 sites periodic, Ne = 8, U/t = 4, 2-site sublattice
    f (16 params) + nearest/next Jastrow + Gutzwiller."""
    return make_problem("ring8_hubbard", chain(8, 1), 8, U=U, sub=(2, 1),
                        jastrow="chain", noise=noise, seed=seed)


def square8_hubbard(noise=0.05, seed=0, U=4.0):
    """8x8 Hubbard, periodic in x / anti-periodic in y, Ne = 64, U/t = 4,
    2x2 sublattice f (256) + distance Jastrow (14) + Gutzwiller (1)."""
    return make_problem("square8_hubbard", square(8, 8, 1, -1), 64, U=U,
                        sub=(2, 2), jastrow="distance", noise=noise, seed=seed)


def square16_hubbard(noise=0.05, seed=0, U=8.0, Ne=224):
    """16x16 Hubbard, anti-periodic in x and y, Ne = 224, U/t = 8, 2x2
    sublattice f (1024) + distance Jastrow (44) + Gutzwiller (1)."""
    return make_problem("square16_hubbard", square(16, 16, -1, -1), Ne, U=U,
                        sub=(2, 2), jastrow="distance", noise=noise, seed=seed)


def square16_hubbard_mlp(hidden=1024, noise=0.05, seed=0, U=8.0, Ne=224):
    """The 16x16 Hubbard workload times an MLP correlation factor
    (512 occupations -> `hidden` tanh units -> one log-amplitude),
    weights initialised N(0, 0.01^2)."""
    return make_problem("square16_hubbard_mlp", square(16, 16, -1, -1), Ne, U=U,
                        sub=(2, 2), jastrow="distance", noise=noise, seed=seed,
                        mlp_hidden=hidden)


def j1j2_heisenberg(L=16, J2=0.5, noise=0.05, seed=0):
    """L x L J1-J2 Heisenberg as a half-filled, doublon-free Hubbard model:
    periodic in x, anti-periodic in y (for the f initialisation), f without
    symmetry reduction, exchange moves only."""
    return make_problem(f"j1j2_{L}x{L}", square(L, L, 1, -1), L * L, t=0.0,
                        J1=1.0, J2=J2, local_spin=True, f_full=True,
                        gutzwiller=False, noise=noise, seed=seed)


def heisenberg_square(L=4, noise=0.05, seed=0, sub=(2, 2)):
    """L x L nearest-neighbour Heisenberg (periodic)."""
    return make_problem(f"heis_{L}x{L}", square(L, L, 1, -1), L * L, t=0.0,
                        J1=1.0, local_spin=True, sub=sub, gutzwiller=False,
                        noise=noise, seed=seed)


def kondo_chain(L=8, t=1.0, J=1.0, bc=1, noise=0.3, seed=0):
    """One-dimensional Kondo lattice: L conduction sites 0..L-1 on a ring
    (hopping t, boundary sign bc on the wrap-around bond) and L local spins
    L..2L-1, local spin L+i coupled to conduction site i by J S.s; Ne = 2L
    (half-filled conduction band).  Local sites carry the per-site
    local-spin constraint; full f with seeded U(-noise, noise) entries,
    Gutzwiller factor on the conduction sites, no Jastrow factor."""
    Ns = 2 * L
    hop_i, hop_j, hop_t = [], [], []
    for i in range(L):
        j = (i + 1) % L
        tij = t * (bc if j < i else 1.0)
        hop_i += [i, j]
        hop_j += [j, i]
        hop_t += [tij, tij]
    f_idx, f_sign, n_f = full_f_layout(Ns)
    g_idx = np.where(np.arange(Ns) < L, 0, -1).astype(np.int32)
    rng = np.random.default_rng(seed)
    params = np.concatenate([[0.0], rng.uniform(-noise, noise, n_f) + 0.5 * np.eye(Ns).reshape(-1)])
    return Problem(name=f"kondo_{L}", lat=Lattice(Ns, 1), Ne=Ns,
                   hop_i=np.array(hop_i, np.int32), hop_j=np.array(hop_j, np.int32),
                   hop_t=np.array(hop_t, np.float64), U=np.zeros(Ns),
                   ex_i=np.arange(L, dtype=np.int32), ex_j=np.arange(L, Ns, dtype=np.int32),
                   ex_J=np.full(L, float(J)), local_spin=False, g_idx=g_idx, n_g=1,
                   v_idx=np.full(Ns * Ns, -1, np.int32), n_v=0, f_idx=f_idx, f_sign=f_sign,
                   n_f=n_f, params=params, p_exchange=0.5,
                   local_sites=np.arange(Ns) >= L)


def batched_hubbard(n_systems=64, seed=0, sizes=(4, 6, 8, 10, 12, 14, 16)):
    """Independent Hubbard systems of uneven size: L drawn from `sizes`,
    filling 0.875 rounded to the nearest even Ne, U/t uniform in [2, 8]."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_systems):
        L = int(sizes[s % len(sizes)])
        Ns = L * L
        Ne = int(round(0.875 * Ns / 2.0)) * 2
        U = float(rng.uniform(2.0, 8.0))
        lat = square(L, L, -1, -1)
        try:
            p = make_problem(f"batch{s}_L{L}", lat, Ne, U=U, sub=(2, 2),
                             jastrow="distance", seed=seed + 1 + s)
        except ValueError:
            lat = square(L, L, 1, -1)
            try:
                p = make_problem(f"batch{s}_L{L}", lat, Ne, U=U, sub=(2, 2),
                                 jastrow="distance", seed=seed + 1 + s)
            except ValueError:
                p = make_problem(f"batch{s}_L{L}", lat, Ne, U=U, sub=(2, 2),
                                 jastrow="distance", seed=seed + 1 + s,
                                 f_init="none", noise=0.5)
        p.meta["U"] = U
        out.append(p)
    return out


def random_samples(n_mc: int, n_p: int, seed: int, density: float = 1.0):
    """Seeded synthetic (E, O) sample arrays for SR parity and timing."""
    rng = np.random.default_rng(seed)
    O = rng.standard_normal((n_mc, n_p))
    if density < 1.0:
        O *= rng.random((n_mc, n_p)) < density
    E = rng.standard_normal(n_mc) + O[:, : min(n_p, 8)].sum(axis=1) * 0.1
    return E, O
