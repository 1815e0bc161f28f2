"""O6: two-site TEBD theta formation with a gate (complex128).

The paper's iTEBD listing (App. A) forms Theta by contracting the MPS
tensors and then applies the two-site evolution operator u with the label
pattern "ijkl","jkmn"->"imnl", i.e. it sums u's *first* two indices.  The
batched workload here uses the explicit formula

    theta[a, s1, s2, b] = sum_{t1, t2, c} G[s1, s2, t1, t2] A[a, t1, c] B[c, t2, b]

which sums G's *last* two indices; the two conventions coincide for a
symmetric gate and ``theta_paper_convention`` provides the paper's one.
"""
from __future__ import annotations

import numpy as np

from .contract import contract


def theta(A, B, G):
    """theta[a,s1,s2,b] (complex128) via two TCI contractions."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    G = np.asarray(G, dtype=np.complex128)
    AB = contract(A, "aic", B, "cjb", "aijb")
    return contract(G, "stij", AB, "aijb", "astb")


def theta_paper_convention(A, B, u):
    """App. A convention: Theta[i,m,n,l] = sum_{j,k} Theta0[i,j,k,l] u[j,k,m,n]."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    AB = contract(A, "aic", B, "cjb", "aijb")
    return contract(AB, "ijkl", np.asarray(u, dtype=np.complex128), "jkmn", "imnl")


def ab_3m(A, B):
    """AB[a,t1,t2,b] by the 3-real-multiplication (3M / Gauss) scheme, float64.

    P1 = Ar Br, P2 = Ai Bi, P3 = (Ar + Ai)(Br + Bi);  Re = P1 - P2, Im = P3 - P1 - P2.
    """
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    p1 = contract(A.real, "aic", B.real, "cjb", "aijb")
    p2 = contract(A.imag, "aic", B.imag, "cjb", "aijb")
    p3 = contract(A.real + A.imag, "aic", B.real + B.imag, "cjb", "aijb")
    return (p1 - p2) + 1j * (p3 - p1 - p2)


def tebd_flops(chis, d: int = 2) -> float:
    """Sum over bonds of 8 chi^3 d^2 + 8 chi^2 d^4 real flops (4M convention)."""
    return float(sum(8.0 * c ** 3 * d * d + 8.0 * c * c * d ** 4 for c in chis))
