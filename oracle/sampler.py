"""Markov-chain Monte Carlo over real-space configurations (Sec. 3.1.1-2).

Moves (Sec. 3.1.2, Fig. update (a), (b)):
* hop: one electron moves to another site (not allowed under the
  local-spin constraint);
* exchange: an up and a down electron on different, singly occupied sites
  swap places.

Proposal distribution (the paper names only the move types; this is the
reading used throughout the project):
* each proposal draws the four Philox words of (walker, counter);
* exchange iff r0 < floor(p_ex * 2^32); hop otherwise;
* hop: electron e = mulhi(r1, Ne), target site = mulhi(r2, Ns); invalid
  (rejected, still counted) if the target already holds that spin, or any
  electron under the local-spin constraint, or if the electron leaves or
  enters a site of the per-site constraint (Kondo local spins, Sec. 4.2:
  they change only by exchange);
* exchange: up electron n = mulhi(r1, N), down electron N + mulhi(r2, N);
  invalid unless the two sites differ, the up site holds no down electron
  and the down site no up electron;
* accept iff u < |psi(x')/psi(x)|^2 with u = (r3 >> 8) 2^-24.
One sweep is Ne proposals.  Electron labels are kept through every move.

The ratio is recomputed from scratch through two full Pfaffians: no fast
update.
"""
import math

import numpy as np

from .fock import from_labels
from .hamiltonian import local_energy
from .philox import exchange_threshold, mulhi, proposal_draw, uniform24


class Chain:
    def __init__(self, wf, ele, seed, system, walker, counter=0, p_exchange=0.0):
        self.wf = wf
        self.Ns = wf.Ns
        self.Ne = len(ele)
        self.N = self.Ne // 2
        self.ele = [int(s) for s in ele]
        self.seed = int(seed)
        self.system = int(system)
        self.walker = int(walker)
        self.counter = int(counter)
        self.thr = exchange_threshold(1.0 if wf.local_spin else p_exchange)
        self.occ = [[-1] * self.Ns, [-1] * self.Ns]
        for k, s in enumerate(self.ele):
            self.occ[1 if k >= self.N else 0][s] = k
        self.n = from_labels(self.ele, self.Ns)
        self.slog = wf.amplitude_slog(self.n)
        if self.slog[0] == 0.0:
            raise ValueError("initial configuration has psi = 0")
        self.n_prop = 0
        self.n_acc = 0

    def _try(self, moves):
        """moves: list of (electron, new site). Returns the new bitmask."""
        n = self.n
        for e, new in moves:
            s = 1 if e >= self.N else 0
            old = self.ele[e]
            n &= ~(1 << (old + self.Ns * s))
            n |= 1 << (new + self.Ns * s)
        return n

    def _apply(self, moves, n_new, slog_new):
        for e, new in moves:
            s = 1 if e >= self.N else 0
            self.occ[s][self.ele[e]] = -1
        for e, new in moves:
            s = 1 if e >= self.N else 0
            self.occ[s][new] = e
            self.ele[e] = new
        self.n = n_new
        self.slog = slog_new

    def propose(self):
        r0, r1, r2, r3 = proposal_draw(self.seed, self.system, self.walker, self.counter)
        self.counter += 1
        self.n_prop += 1
        u = uniform24(r3)
        if r0 < self.thr:
            a = mulhi(r1, self.N)
            b = self.N + mulhi(r2, self.N)
            i, j = self.ele[a], self.ele[b]
            if i == j or self.occ[1][i] >= 0 or self.occ[0][j] >= 0:
                return False
            moves = [(a, j), (b, i)]
        else:
            e = mulhi(r1, self.Ne)
            t = mulhi(r2, self.Ns)
            s = 1 if e >= self.N else 0
            if self.occ[s][t] >= 0:
                return False
            if self.wf.local_spin and self.occ[1 - s][t] >= 0:
                return False
            if self.wf.local_sites is not None and (self.wf.local_sites[t] or
                                                    self.wf.local_sites[self.ele[e]]):
                return False
            moves = [(e, t)]
        n_new = self._try(moves)
        slog_new = self.wf.amplitude_slog(n_new)
        if slog_new[0] == 0.0:
            return False
        if u < math.exp(2.0 * (slog_new[1] - self.slog[1])):
            self._apply(moves, n_new, slog_new)
            self.n_acc += 1
            return True
        return False

    def sweeps(self, k):
        for _ in range(k * self.Ne):
            self.propose()


def run_sampling(wf, ele0, seed, system, n_warmup, n_samples, sweeps_between,
                 p_exchange, counters=None, measure=True):
    """Sample every walker: n_warmup sweeps, then n_samples times
    (sweeps_between sweeps, measure).  Returns a dict with E [W*S],
    O [W*S, Np] (row = walker * n_samples + sample), final configurations,
    counters and acceptance counts."""
    W = len(ele0)
    Np = wf.params.size
    E = np.zeros(W * n_samples)
    O = np.zeros((W * n_samples, Np))
    ele_out = np.zeros_like(np.asarray(ele0))
    ctr_out = np.zeros(W, np.int64)
    n_prop = n_acc = 0
    for w in range(W):
        ch = Chain(wf, ele0[w], seed, system, w,
                   0 if counters is None else int(counters[w]), p_exchange)
        ch.sweeps(n_warmup)
        for s in range(n_samples):
            ch.sweeps(sweeps_between)
            if measure:
                E[w * n_samples + s] = local_energy(wf, ch.n)
                O[w * n_samples + s] = wf.log_derivatives(ch.n)
        ele_out[w] = ch.ele
        ctr_out[w] = ch.counter
        n_prop += ch.n_prop
        n_acc += ch.n_acc
    return dict(E=E, O=O, ele=ele_out, counters=ctr_out, n_prop=n_prop, n_acc=n_acc)
