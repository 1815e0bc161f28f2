"""iTEBD ground-state iteration of the paper's App. A, written out (test infrastructure only).

What the App. A program computes, restated: the imaginary-time gate
u = exp(-dt h) of the two-site term (from the eigendecomposition of h, then
reshaped u[s1, s2, t1, t2]); a two-site unit cell Gamma_A, Lambda_A,
Gamma_B, Lambda_B.  Iteration i uses A = i mod 2, B = (i + 1) mod 2:

    Theta[i, j, k, l] = LB[i] Gamma_A[i, j, a] LA[a] Gamma_B[a, k, b] LB[b]   (b = l)
    Theta'[i, m, n, l] = sum_{j k} Theta[i, j, k, l] u[j, k, m, n]
    Gamma_A, Lambda_A, Gamma_B <- trunc_svd(Theta', 2 row bonds, chi, s_min)
    Lambda_A /= ||Lambda_A||
    Gamma_A[i, :, :] /= LB[i];  Gamma_B[:, :, k] /= LB[k]
    E_i = -log(sum Theta'^2) / (2 dt)

(LA, LB: the current Lambda_A, Lambda_B.)  E_i estimates the energy per bond,
which is the energy per site of the infinite chain.
"""
from __future__ import annotations

import numpy as np

from .contract import contract
from .linalg import trunc_svd


def gate(h, dt: float, d: int = 2):
    w, v = np.linalg.eigh(np.asarray(h, dtype=np.float64))
    return (v @ np.diag(np.exp(-dt * w)) @ v.T).reshape(d, d, d, d)


def itebd(h, dt: float, gammas, lambdas, chi: int, niters: int, s_min: float = 1e-10):
    """Return (energies per iteration, final gammas, final lambdas)."""
    u = gate(h, dt)
    G = [np.array(g, dtype=np.float64) for g in gammas]
    Lm = [np.array(l, dtype=np.float64) for l in lambdas]
    energies = []
    for i in range(niters):
        A, B = i % 2, (i + 1) % 2
        LA, LB = np.diag(Lm[A]), np.diag(Lm[B])
        th = contract(LB, "ij", G[A], "jkl", "ikl")
        th = contract(th, "ijk", LA, "kl", "ijl")
        th = contract(th, "ijk", G[B], "klm", "ijlm")
        th = contract(th, "ijkl", LB, "lm", "ijkm")
        th = contract(th, "ijkl", u, "jkmn", "imnl")
        uA, sA, vB, _ = trunc_svd(th, 2, 1, chi, 0.0, s_min)
        sA = sA / np.linalg.norm(sA)
        inv = np.diag(1.0 / Lm[B])
        G[A] = contract(inv, "ij", uA, "jkl", "ikl")
        G[B] = contract(vB, "ijk", inv, "kl", "ijl")
        Lm[A] = sA
        energies.append(-np.log(np.sum(th * th)) / dt / 2.0)
    return energies, G, Lm


def tfim_exact_energy(J: float, g: float) -> float:
    """Ground energy per site of H = J sum ZZ - g sum X on the infinite chain (Pfeuty 1970):
    -(1/pi) int_0^pi sqrt(J^2 + g^2 + 2 J g cos k) dk (the sign of J does not matter)."""
    from scipy.integrate import quad
    val, _ = quad(lambda k: np.sqrt(J * J + g * g + 2.0 * J * g * np.cos(k)), 0.0, np.pi, epsabs=1e-14, epsrel=1e-14)
    return -val / np.pi
