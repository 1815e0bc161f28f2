"""O5: U(1) block-sparse H_eff via densification.

The paper lists symmetric (block-sparse) tensors as future work (Sec. IV);
the block-sparse effective Hamiltonian is defined as the dense one applied
to the zero-filled (densified) tensors, so the dense O3 result restricted
to the allowed blocks *is* the block-sparse result.
"""
from __future__ import annotations

import numpy as np

from .heff import heff_apply


def _offsets(dims):
    return np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(np.int64)


def densify_env(blocks: dict, dims, Dw: int = 5):
    """E[x, w, x'] dense from blocks keyed (ix, w, ix') of shape [dims[ix], dims[ix']]."""
    off = _offsets(dims)
    n = int(np.sum(dims))
    E = np.zeros((n, Dw, n))
    for (i, w, j), blk in blocks.items():
        E[off[i]:off[i] + dims[i], w, off[j]:off[j] + dims[j]] = blk
    return E


def densify_psi(blocks: dict, dims, d: int = 2):
    """psi[a', t1, t2, b'] dense from blocks keyed (ia', t1, t2, ib')."""
    off = _offsets(dims)
    n = int(np.sum(dims))
    P = np.zeros((n, d, d, n))
    for (i, t1, t2, j), blk in blocks.items():
        P[off[i]:off[i] + dims[i], t1, t2, off[j]:off[j] + dims[j]] = blk
    return P


def extract_blocks(dense_out, keys, dims):
    """Blocks (ia, s1, s2, ib) of a dense out[a, s1, s2, b]."""
    off = _offsets(dims)
    return {k: dense_out[off[k[0]]:off[k[0]] + dims[k[0]], k[1], k[2], off[k[3]]:off[k[3]] + dims[k[3]]].copy()
            for k in keys}


def bs_heff_apply(inp: dict):
    """Block-sparse H_eff . psi: returns (blocks keyed like psi, dense result)."""
    dims = inp["dims"]
    L = densify_env({k: v.astype(np.float64) for k, v in inp["L"].items()}, dims)
    R = densify_env({k: v.astype(np.float64) for k, v in inp["R"].items()}, dims)
    P = densify_psi({k: v.astype(np.float64) for k, v in inp["psi"].items()}, dims)
    out = heff_apply(L, inp["W"], R, P, order="R")
    return extract_blocks(out, list(inp["psi"].keys()), dims), out


def bs_flops(inp: dict) -> float:
    """Algorithmic flops of the block-sparse matvec: 2 m n k over every nonzero block product.

    Counted from the block lists (not the dense 6.9e11): GEMM1 pairs each psi
    block (a', t1, t2, b') with each R block (b, wr, b'); GEMM2 pairs each L
    block (a, wl, a') with each V block (s1, s2, b, wl, a') that exists, i.e.
    q_b = q_a + c(s1) + c(s2); the W-application costs 2 d^4 Dw^2 per (a', b)
    element pair that carries a nonzero U block.
    """
    dims = inp["dims"]
    qmax = inp["qmax"]
    nsec = len(dims)
    psi_keys = list(inp["psi"].keys())
    R_keys = list(inp["R"].keys())
    L_keys = list(inp["L"].keys())
    W = inp["W"]
    d = W.shape[2]
    phys = np.array([+1, -1])
    fl = 0.0
    # GEMM1: U(a',t1,t2,b,wr) = psi(a',t1,t2,b') R(b,wr,b')^T
    ublocks = set()
    for (ia, t1, t2, ib) in psi_keys:
        for (jb, wr, jbp) in R_keys:
            if jbp == ib:
                fl += 2.0 * dims[ia] * dims[jb] * dims[ib]
                ublocks.add((ia, jb))
    # W application on every (a', b) sector pair that carries U
    for (ia, jb) in ublocks:
        fl += 2.0 * dims[ia] * dims[jb] * (d ** 4) * (W.shape[0] ** 2)
    # GEMM2: out(a,s1,s2,b) = sum_{wl, a'} L(a,wl,a') V(s1,s2,b,wl,a')
    for ia in range(nsec):
        qa = ia - qmax
        for s1 in range(d):
            for s2 in range(d):
                ib = qa + phys[s1] + phys[s2] + qmax
                if not (0 <= ib < nsec):
                    continue
                for (ja, wl, jap) in L_keys:
                    if ja == ia and (jap, ib) in ublocks:
                        fl += 2.0 * dims[ia] * dims[ib] * dims[jap]
    return fl
