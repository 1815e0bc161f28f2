"""Belief-propagation message update on a TNS norm network (App. B), written out.

Test infrastructure only.  App. B regauges a tensor-network state by BP on
its norm network <psi|psi> (the scheme of Tindall & Fishman, SciPost Phys.
15, 222 (2023)): every directed bond i -> j carries a message M_{i->j}, a
matrix over (ket bond index, bra bond index), and a BP iteration replaces
each message by the norm network's site i (V_i and its copy, physical index
summed) contracted with the messages that enter i from every neighbour
except j:

    M_{i->j}[b, b'] = sum V_i[s, .., b, ..] V_i[s, .., b', ..] prod_{k != j} M_{k->i}[b_k, b_k']

normalised to unit Frobenius norm.  The update is synchronous (all new
messages from the previous set), so messages are local and independent
within an iteration.  Bond order of V_i: physical index first, then one bond
per neighbour in ascending neighbour order.  Messages are indexed per edge
e = (u, v): 2e is u -> v, 2e + 1 is v -> u.

Readings (the paper's figure states the fixed-point relation, not the
normalisation or schedule): Frobenius normalisation, synchronous schedule,
residual = max over messages of ||M_new - M_old||_F.
"""
from __future__ import annotations

import numpy as np

from .contract import contract

KET = "abcdefgh"
BRA = "ABCDEFGH"


def neighbours(n: int, edges):
    nb = [[] for _ in range(n)]
    for e, (u, v) in enumerate(edges):
        nb[u].append((v, 2 * e + 1))   # message v -> u enters u
        nb[v].append((u, 2 * e))       # message u -> v enters v
    return [sorted(x) for x in nb]


def message_update(V_i, incoming, out_pos: int):
    """New (unnormalised) message leaving site i through its bond at position out_pos.

    incoming[q]: message entering i through bond q (None for q == out_pos)."""
    k = V_i.ndim - 1
    ket = "s" + KET[:k]
    cur = list(ket)
    T = V_i
    for q in range(k):
        if q == out_pos:
            continue
        nxt = cur.copy()
        nxt[1 + q] = BRA[q]
        T = contract(T, "".join(cur), incoming[q], KET[q] + BRA[q], "".join(nxt))
        cur = nxt
    bra = "s" + "".join(BRA[q] for q in range(k))
    return contract(T, "".join(cur), V_i, bra, KET[out_pos] + BRA[out_pos])


def bp_iteration(n: int, edges, V, M):
    """One synchronous BP iteration; returns (new messages, residual)."""
    nb = neighbours(n, edges)
    new = [None] * len(M)
    for e, (u, v) in enumerate(edges):
        for src, dst, idx in ((u, v, 2 * e), (v, u, 2 * e + 1)):
            bonds = nb[src]
            incoming = [M[m_in] for (_, m_in) in bonds]
            out_pos = [w for (w, _) in bonds].index(dst)
            m = message_update(V[src], incoming, out_pos)
            new[idx] = m / np.linalg.norm(m)
    res = max((np.linalg.norm(a - b) for a, b in zip(new, M)), default=0.0)
    return new, res


def bp(n: int, edges, V, M, niters: int, tol: float = 0.0):
    """Up to niters iterations, stopping once the residual is <= tol; returns (messages, residuals)."""
    res = []
    for _ in range(niters):
        M, r = bp_iteration(n, edges, V, M)
        res.append(r)
        if r <= tol:
            break
    return M, res


def site_density(n: int, edges, V, M, i: int):
    """Reduced density matrix of site i from the BP environment, trace 1."""
    nb = neighbours(n, edges)
    k = V[i].ndim - 1
    ket = "s" + KET[:k]
    cur = list(ket)
    T = V[i]
    for q, (_, m_in) in enumerate(nb[i]):
        nxt = cur.copy()
        nxt[1 + q] = BRA[q]
        T = contract(T, "".join(cur), M[m_in], KET[q] + BRA[q], "".join(nxt))
        cur = nxt
    rho = contract(T, "".join(cur), V[i], "t" + "".join(BRA[q] for q in range(k)), "st")
    return rho / np.trace(rho)
