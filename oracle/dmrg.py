"""Two-site finite DMRG around the H_eff matvec, written out (test infrastructure only).

The paper names DMRG as a target of TCI (Sec. I) without spelling it out; the
algorithm is the textbook two-site sweep (Schollwoeck, Ann. Phys. 326, 96
(2011), Secs. 6.2-6.4) expressed with TCI ``contract``, the oracle H_eff,
Lanczos and ``trunc_svd``:

* start: the Neel product state, A_k[0, k mod 2, 0] = 1 (bond dimension 1),
  trivially in canonical form; boundary environments L[0, Dw-1, 0] = 1 and
  R[0, 0, 0] = 1 (the MPO's left vector selects its last channel, the right
  vector its first);
* right environments R_k (sites k..N-1) built from the right end;
* each sweep: bonds (k, k+1) for k = 0..N-2 (left to right) then
  k = N-2..0 (right to left).  At a bond: psi = A_k A_{k+1}; the lowest
  eigenpair of H_eff(L_k, W, W, R_{k+2}) by Lanczos started from psi;
  trunc_svd(psi, 2 row bonds, chi_min 1, chi_max, target 0, s_min);
  moving right A_k = U, A_{k+1} = S V^T and L_{k+1} from L_k and A_k;
  moving left A_{k+1} = V^T, A_k = U S and R_{k+1} from R_{k+2} and A_{k+1};
* the energy of a sweep is the Ritz value of its last bond.

Environment updates (A real):
    L_{k+1}[b, w', b'] = sum A_k[a, s, b] L_k[a, w, a'] W[w, w', s, t] A_k[a', t, b']
    R_{k}[a, w, a']    = sum A_k[a, s, b] W[w, w', s, t] R_{k+1}[b, w', b'] A_k[a', t, b']
"""
from __future__ import annotations

import numpy as np

from .contract import contract
from .heff import heff_apply
from .lanczos import lanczos
from .linalg import trunc_svd


def update_left(L, A, W):
    T = contract(L, "awx", A, "xty", "awty")
    T = contract(T, "awty", W, "wvst", "avsy")
    return contract(A, "asb", T, "avsy", "bvy")


def update_right(R, A, W):
    T = contract(R, "bvy", A, "xty", "bvxt")
    T = contract(T, "bvxt", W, "wvst", "bwsx")
    return contract(A, "asb", T, "bwsx", "awx")


def neel_mps(nsites: int, d: int = 2):
    mps = []
    for k in range(nsites):
        A = np.zeros((1, d, 1))
        A[0, k % 2, 0] = 1.0
        mps.append(A)
    return mps


def dmrg(W, nsites: int, chi_max: int, nsweeps: int, lanczos_steps: int = 20, s_min: float = 1e-12):
    """Return (energies per sweep, largest truncation error of each sweep)."""
    W = np.asarray(W, dtype=np.float64)
    Dw = W.shape[0]
    A = neel_mps(nsites)
    L = [None] * (nsites + 1)
    R = [None] * (nsites + 2)
    L[0] = np.zeros((1, Dw, 1))
    L[0][0, Dw - 1, 0] = 1.0
    R[nsites] = np.zeros((1, Dw, 1))
    R[nsites][0, 0, 0] = 1.0
    for k in range(nsites - 1, 0, -1):
        R[k] = update_right(R[k + 1], A[k], W)
    energies, errs = [], []

    def solve(k):
        psi = contract(A[k], "abc", A[k + 1], "cde", "abde")
        mv = lambda v: heff_apply(L[k], W, R[k + 2], v.reshape(psi.shape))
        res = lanczos(mv, psi, lanczos_steps)
        return res["theta"], res["x"].reshape(psi.shape)

    for _ in range(nsweeps):
        e = 0.0
        terr = 0.0
        for k in range(nsites - 1):                       # left to right
            e, psi = solve(k)
            u, s, vt, err = trunc_svd(psi, 2, 1, chi_max, 0.0, s_min)
            terr = max(terr, err)
            A[k] = u
            A[k + 1] = contract(np.diag(s), "ab", vt, "bcd", "acd")
            L[k + 1] = update_left(L[k], A[k], W)
        for k in range(nsites - 2, -1, -1):               # right to left
            e, psi = solve(k)
            u, s, vt, err = trunc_svd(psi, 2, 1, chi_max, 0.0, s_min)
            terr = max(terr, err)
            A[k + 1] = vt
            A[k] = contract(u, "abc", np.diag(s), "cd", "abd")
            R[k + 1] = update_right(R[k + 2], A[k + 1], W)
        energies.append(e)
        errs.append(terr)
    return energies, errs
