"""O2/O3: Heisenberg MPO helpers and the two-site DMRG effective Hamiltonian.

The paper names DMRG only as a target application of TCI (Sec. I); the
effective Hamiltonian below is the textbook two-site one (Schollwoeck,
Ann. Phys. 326, 96 (2011), Sec. 6), written with TCI ``contract`` calls:

    out[a, s1, s2, b] = sum L[a, wl, a'] W[wl, wm, s1, t1] W[wm, wr, s2, t2]
                            R[b, wr, b'] psi[a', t1, t2, b']

L[a, w, a'] (bra a, ket a'), R[b, w, b'] (bra b, ket b'), W[wl, wr, s, t]
(s bra, t ket).  Two independent contraction orders are provided (L first,
R first) and an explicit dense matrix for tiny bond dimensions.
"""
from __future__ import annotations

import numpy as np

from .contract import contract


def heff_apply(L, W, R, psi, order: str = "R", W2=None):
    """H_eff . psi in float64 as four pairwise contractions.

    W acts on the left site, W2 (default: W) on the right one.
    order="L": (L psi) W W2 R;  order="R": (psi R) W2 W L.
    Labels: a/x = bra/ket left bond, b/y = bra/ket right bond, w/m/r = MPO
    bonds (left, middle, right), s/u = bra physical, i/j = ket physical.
    """
    W2 = W if W2 is None else W2
    if order == "L":
        T = contract(L, "awx", psi, "xijy", "awijy")
        T = contract(T, "awijy", W, "wmsi", "amsjy")
        T = contract(T, "amsjy", W2, "mruj", "asury")
        return contract(T, "asury", R, "bry", "asub")
    if order == "R":
        U = contract(psi, "xijy", R, "bry", "xijbr")
        U = contract(U, "xijbr", W2, "mruj", "xibmu")
        U = contract(U, "xibmu", W, "wmsi", "xbusw")
        return contract(L, "awx", U, "xbusw", "asub")
    raise ValueError(order)


def heff_rows(L, W, R, psi, rows):
    """out[a, :, :, :] for the selected left indices a only (sampling at large chi).

    Same sum as ``heff_apply`` restricted to a in ``rows``; cost per row is
    O(Dw chi^2 d^2) instead of O(Dw chi^3 d^2).
    """
    rows = np.asarray(rows, dtype=np.int64)
    return heff_apply(L[rows], W, R, psi, order="L")


def heff_matrix_loops(L, W, R, W2=None):
    """Dense H_eff[(a,s1,s2,b), (a',t1,t2,b')] by explicit loops (chi <= 3); W2 (default W) on the right site."""
    W2 = W if W2 is None else W2
    chi_l, Dw, _ = L.shape
    chi_r = R.shape[0]
    d = W.shape[2]
    n = chi_l * d * d * chi_r
    H = np.zeros((n, n), dtype=np.result_type(L, W, W2, R))

    def idx(a, s1, s2, b):
        return ((a * d + s1) * d + s2) * chi_r + b

    for a in range(chi_l):
        for s1 in range(d):
            for s2 in range(d):
                for b in range(chi_r):
                    for ap in range(chi_l):
                        for t1 in range(d):
                            for t2 in range(d):
                                for bp in range(chi_r):
                                    acc = 0.0
                                    for wl in range(Dw):
                                        for wm in range(Dw):
                                            for wr in range(Dw):
                                                acc += (L[a, wl, ap] * W[wl, wm, s1, t1]
                                                        * W2[wm, wr, s2, t2] * R[b, wr, bp])
                                    H[idx(a, s1, s2, b), idx(ap, t1, t2, bp)] = acc
    return H


def heff_flops(chi_l: int, chi_r: int | None = None, d: int = 2, Dw: int = 5) -> float:
    """Algorithmic flops of one dense matvec: 4 chi^3 d^2 Dw + 2 chi^2 d^4 Dw^2 (chi_l = chi_r)."""
    chi_r = chi_l if chi_r is None else chi_r
    # (psi R): 2 * chi_l d^2 * chi_r Dw * chi_r ; (.. L): 2 * chi_l * d^2 chi_r * Dw chi_l
    g1 = 2.0 * chi_l * d * d * chi_r * Dw * chi_r
    g2 = 2.0 * chi_l * d * d * chi_r * Dw * chi_l
    ww = 2.0 * chi_l * chi_r * (d ** 4) * Dw * Dw
    return g1 + g2 + ww


# ---------------------------------------------------------------------------
# Exact environments of a full-rank computational-basis MPS (pins O3 iv)
# ---------------------------------------------------------------------------
def left_env(W, nsites: int):
    """L over ``nsites`` sites: L_0[0,w,0] = delta_{w,Dw-1}; L_{k+1}[(a,s),w',(a',t)] = sum_w L_k W."""
    Dw, d = W.shape[0], W.shape[2]
    Lk = np.zeros((1, Dw, 1))
    Lk[0, Dw - 1, 0] = 1.0
    for _ in range(nsites):
        n = Lk.shape[0]
        T = contract(Lk, "awx", W, "wvst", "asvxt")      # [a, s, w', a', t]
        Lk = T.reshape(n * d, Dw, n * d)
    return Lk


def right_env(W, nsites: int):
    """R over ``nsites`` sites: R_0[0,w,0] = delta_{w,0}; R_{k+1}[(s,b),w,(t,b')] = sum_w' W R_k."""
    Dw, d = W.shape[0], W.shape[2]
    Rk = np.zeros((1, Dw, 1))
    Rk[0, 0, 0] = 1.0
    for _ in range(nsites):
        n = Rk.shape[0]
        T = contract(W, "wvst", Rk, "bvy", "sbwty")       # [s, b, w, t, b']
        Rk = T.reshape(d * n, Dw, d * n)
    return Rk


def mpo_chain_matrix(W, nsites: int):
    """Full operator of an ``nsites`` MPO chain (boundaries wl = Dw-1, wr = 0)."""
    Dw, d = W.shape[0], W.shape[2]
    # M[w, (s...), (t...)] accumulated site by site from the left boundary.
    M = np.zeros((Dw, 1, 1))
    M[Dw - 1, 0, 0] = 1.0
    for _ in range(nsites):
        n = M.shape[1]
        T = contract(M, "wab", W, "wvst", "vasbt")         # [w', a, s, b, t]
        M = T.reshape(Dw, n * d, n * d)
    return M[0]
