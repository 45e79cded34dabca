"""Stochastic reconfiguration (Sec. 3.3.1-3.3.2, Algorithm 1).

* S_km = <O_k O_m> - <O_k><O_m>, g_m = <H O_m> - <H><O_m> (real parameters,
  so Re is the identity), averages over the N_MC samples (Eq. MC).
* Diagonal shift (the paper gives no form): S~_kk = S_kk (1 + shift_rel)
  + shift_abs.
* Delta alpha = -dtau S~^-1 g (Eq. SR_equation_system).
* Solve by Cholesky S~ = L L^T (Sec. 3.3.2, first paragraph) or by CG
  (Algorithm 1) whose matrix-vector product is the SR-CG form of Sec. 3.3.2:
  y = z1 - z2 with z1 = (1/N_MC) O^T (O v) and z2 = <O> (<O> . v), O the
  uncentred sample matrix.
"""
import numpy as np


def sr_matrices(E, O, weights=None):
    """S, g, <O>, <E> of Sec. 3.3.1 for real parameters.

    <A> is the sample mean over the N_MC rows (Eq. MC), or, with `weights`
    (one non-negative weight per row, normalised here), the weighted mean
    sum_u w_u A_u: exact enumeration passes rho(x) = |psi(x)|^2 / <psi|psi>
    and so obtains the exact S and g from this same function."""
    E = np.asarray(E, np.float64)
    O = np.asarray(O, np.float64)
    if weights is None:
        w = np.full(E.size, 1.0 / E.size)
    else:
        w = np.asarray(weights, np.float64)
        w = w / w.sum()
    obar = w @ O
    ebar = float(w @ E)
    S = (O * w[:, None]).T @ O - np.outer(obar, obar)
    g = (O * w[:, None]).T @ E - ebar * obar
    return S, g, obar, ebar


def shifted(S, shift_rel=0.0, shift_abs=0.0):
    St = S.copy()
    St[np.diag_indices_from(St)] = np.diag(S) * (1.0 + shift_rel) + shift_abs
    return St


def solve_cholesky(St, g):
    L = np.linalg.cholesky(St)
    from scipy.linalg import solve_triangular
    y = solve_triangular(L, g, lower=True)
    return solve_triangular(L.T, y, lower=False)


def srcg_matvec(O, obar, diagS, v, shift_rel=0.0, shift_abs=0.0):
    """S~ v without forming S: 2(N_MC + 1) N_p products for the S part."""
    nmc = O.shape[0]
    z1 = O.T @ (O @ v) / nmc
    z2 = obar * (obar @ v)
    return z1 - z2 + (shift_rel * diagS + shift_abs) * v


def cg(matvec, b, x0=None, eps=1e-10, kmax=1000):
    """Algorithm 1: CG for A x = b; stops when |r|^2 < eps^2 |b|^2.
    Returns (x, iterations)."""
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    thr = eps * eps * float(b @ b)
    r = b - matvec(x)
    p = r.copy()
    rho = float(r @ r)
    it = 0
    if rho < thr:
        return x, 0
    for it in range(1, kmax + 1):
        w = matvec(p)
        alpha = rho / float(p @ w)
        x = x + alpha * p
        r = r - alpha * w
        rho_new = float(r @ r)
        if rho_new < thr:
            break
        p = r + (rho_new / rho) * p
        rho = rho_new
    return x, it


def sr_step(E, O, dtau, shift_rel=0.0, shift_abs=0.0, solver="cholesky",
            cg_eps=1e-10, cg_kmax=1000):
    """Return (delta_alpha, info) for one SR step."""
    S, g, obar, ebar = sr_matrices(E, O)
    if solver == "cholesky":
        x = solve_cholesky(shifted(S, shift_rel, shift_abs), g)
        it = 0
    else:
        O64 = np.asarray(O, np.float64)
        diagS = np.diag(S).copy()
        x, it = cg(lambda v: srcg_matvec(O64, obar, diagS, v, shift_rel, shift_abs),
                   g, eps=cg_eps, kmax=cg_kmax)
    return -dtau * x, dict(S=S, g=g, obar=obar, ebar=ebar, cg_iters=it)
