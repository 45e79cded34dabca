"""psi(x) = <x| P_G P_J |phi_AP-Pf> for real parameters, and the
log-derivatives O_k(x) = d ln<x|psi> / d alpha_k.

* Pair-product part (Sec. 3.2.1, Eqs. Pf and AP-Pf): F_{(a up),(b down)} =
  f_ab, all other F_IJ = 0; <x|phi> = (Ne/2)! Pf(X) with
  X_IJ = F_IJ - F_JI over the occupied orbitals in ascending order.
* Correlation factors (Sec. 3.2.3): P_G = exp(sum_i g_i n_i,up n_i,dn),
  P_J = exp(1/2 sum_{i != j} v_ij (n_i - 1)(n_j - 1)).  Under the
  local-spin constraint (g -> -infinity, Sec. 3.2.3) a doubly occupied site
  gives psi = 0.  With a per-site constraint (local spins of the Kondo
  lattice, Sec. 4.2: double occupancy excluded on those sites) psi = 0
  unless each marked site holds exactly one electron.
* O_k (Sec. 3.3.1): Gutzwiller O = D_k(x); Jastrow O = sum over the class
  of (n_i - 1)(n_j - 1) for i < j; pair orbital dPf/dF_AB = -Pf(X) (X^-1)_AB
  (Eq. DiffPf and Appendix C), summed over the class with the class sign.
* Optional learned correlation factor (not in the paper): an MLP on the
  spin-resolved occupations n (n_c, c = i + Ns*sigma), multiplying psi by
  exp(w2 . tanh(W1 n + b1) + b2); its O_k are the derivatives of that
  exponent: dW1_kc = w2_k (1 - tanh^2 h_k) n_c, db1_k = w2_k (1 - tanh^2 h_k),
  dw2_k = tanh h_k, db2 = 1.
"""
import math

import numpy as np

from .fock import occupied
from .pfaffian import pfaffian_slog


class Wavefunction:
    def __init__(self, prob, params=None):
        p = np.asarray(prob.params if params is None else params, np.float64)
        self.prob = prob
        self.params = p
        Ns = self.Ns = int(prob.lat.Ns)
        self.Ne = int(prob.Ne)
        self.n_g, self.n_v, self.n_f = int(prob.n_g), int(prob.n_v), int(prob.n_f)
        self.local_spin = bool(prob.local_spin)
        ls = getattr(prob, "local_sites", None)
        self.local_sites = None if ls is None else np.asarray(ls, bool).reshape(Ns)
        gi = np.asarray(prob.g_idx).reshape(Ns)
        self.g_site = np.where(gi >= 0, p[np.maximum(gi, 0)], 0.0) if self.n_g else np.zeros(Ns)
        vi = np.asarray(prob.v_idx).reshape(Ns, Ns)
        pv = p[self.n_g:self.n_g + self.n_v]
        self.v = np.where(vi >= 0, pv[np.maximum(vi, 0)] if self.n_v else 0.0, 0.0)
        fi = np.asarray(prob.f_idx).reshape(Ns, Ns)
        fs = np.asarray(prob.f_sign).reshape(Ns, Ns).astype(np.float64)
        pf = p[self.n_g + self.n_v:self.n_g + self.n_v + self.n_f]
        self.f = np.where(fi >= 0, pf[np.maximum(fi, 0)], 0.0) * fs
        F = np.zeros((2 * Ns, 2 * Ns))
        F[:Ns, Ns:] = self.f
        self.F = F
        self.n_h = int(getattr(prob, "n_hidden", 0) or 0)
        if self.n_h:
            H, C = self.n_h, 2 * Ns
            b = self.n_g + self.n_v + self.n_f
            self.W1 = p[b:b + H * C].reshape(H, C)
            self.b1 = p[b + H * C:b + H * C + H]
            self.w2 = p[b + H * C + H:b + H * C + 2 * H]
            self.b2 = float(p[b + H * C + 2 * H])

    def occ_vector(self, n):
        up, dn = self.occ(n)
        return np.concatenate([up, dn])

    def mlp_log(self, n):
        """w2 . tanh(W1 n + b1) + b2 (0 without the MLP factor)."""
        if not self.n_h:
            return 0.0
        h = self.W1 @ self.occ_vector(n) + self.b1
        return float(self.w2 @ np.tanh(h) + self.b2)

    # -- configuration helpers -------------------------------------------
    def occ(self, n):
        Ns = self.Ns
        up = np.array([(n >> i) & 1 for i in range(Ns)], np.float64)
        dn = np.array([(n >> (Ns + i)) & 1 for i in range(Ns)], np.float64)
        return up, dn

    def X(self, n):
        orbs = occupied(n, 2 * self.Ns)
        Fs = self.F[np.ix_(orbs, orbs)]
        return Fs - Fs.T, orbs

    # -- amplitude -------------------------------------------------------
    def log_correlation(self, n):
        up, dn = self.occ(n)
        m = up + dn - 1.0
        return float(self.g_site @ (up * dn) + 0.5 * m @ self.v @ m)

    def amplitude_slog(self, n):
        """(sign, log|<x|psi>|) including the (Ne/2)! factor."""
        up, dn = self.occ(n)
        if self.local_spin and np.any(up * dn):
            return 0.0, -math.inf
        if self.local_sites is not None and np.any((up + dn)[self.local_sites] != 1):
            return 0.0, -math.inf
        X, _ = self.X(n)
        s, l = pfaffian_slog(X)
        if s == 0.0:
            return 0.0, -math.inf
        return s, l + math.lgamma(self.Ne // 2 + 1) + self.log_correlation(n) + self.mlp_log(n)

    def amplitude(self, n):
        s, l = self.amplitude_slog(n)
        return s * math.exp(l) if s != 0.0 else 0.0

    def ratio(self, n_new, n_old):
        """<x'|psi> / <x|psi> in the canonical basis."""
        s1, l1 = self.amplitude_slog(n_new)
        s0, l0 = self.amplitude_slog(n_old)
        if s0 == 0.0:
            raise ZeroDivisionError("psi(x) = 0")
        if s1 == 0.0:
            return 0.0
        return s1 * s0 * math.exp(l1 - l0)

    # -- log-derivatives -------------------------------------------------
    def log_derivatives(self, n):
        """O_k(x) for all parameters, analytic (Sec. 3.3.1, Appendix C)."""
        Ns = self.Ns
        up, dn = self.occ(n)
        out = np.zeros(self.params.size)
        # Gutzwiller: d/dg_k of sum_i g_i D_i = number of doublons in class k.
        gi = np.asarray(self.prob.g_idx).reshape(Ns)
        for i in range(Ns):
            if gi[i] >= 0 and self.n_g:
                out[gi[i]] += up[i] * dn[i]
        # Jastrow: sum over unordered pairs in the class.
        if self.n_v:
            vi = np.asarray(self.prob.v_idx).reshape(Ns, Ns)
            m = up + dn - 1.0
            for i in range(Ns):
                for j in range(i + 1, Ns):
                    if vi[i, j] >= 0:
                        out[self.n_g + vi[i, j]] += m[i] * m[j]
        # Pair orbital: d ln Pf / dF_AB = -(X^-1)_AB.
        X, orbs = self.X(n)
        Xinv = np.linalg.inv(X)
        pos = {I: k for k, I in enumerate(orbs)}
        fi = np.asarray(self.prob.f_idx).reshape(Ns, Ns)
        fs = np.asarray(self.prob.f_sign).reshape(Ns, Ns)
        base = self.n_g + self.n_v
        for a in range(Ns):
            if a not in pos:
                continue
            for b in range(Ns):
                B = Ns + b
                if B not in pos or fi[a, b] < 0:
                    continue
                out[base + fi[a, b]] += fs[a, b] * (-Xinv[pos[a], pos[B]])
        if self.n_h:
            H, C = self.n_h, 2 * Ns
            nv = self.occ_vector(n)
            t = np.tanh(self.W1 @ nv + self.b1)
            d = self.w2 * (1.0 - t * t)
            b = self.n_g + self.n_v + self.n_f
            out[b:b + H * C] = np.outer(d, nv).reshape(-1)
            out[b + H * C:b + H * C + H] = d
            out[b + H * C + H:b + H * C + 2 * H] = t
            out[b + H * C + 2 * H] = 1.0
        return out

    def log_derivatives_fd(self, n, h=1e-6):
        """Central finite differences of ln|<x|psi>| (self-check)."""
        out = np.zeros_like(self.params)
        for k in range(self.params.size):
            pp = self.params.copy()
            pm = self.params.copy()
            pp[k] += h
            pm[k] -= h
            lp = Wavefunction(self.prob, pp).amplitude_slog(n)[1]
            lm = Wavefunction(self.prob, pm).amplitude_slog(n)[1]
            out[k] = (lp - lm) / (2 * h)
        return out
