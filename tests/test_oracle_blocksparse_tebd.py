"""Pins for oracles O5 (block-sparse), O6 (TEBD theta) and O7 (precision model)."""
import numpy as np
import pytest

from oracle import blocksparse, heff, precision, tebd
from oracle.contract import contract, contract_bruteforce, rel_frob_err
from tci_synth import (MPO_CHANNEL_CHARGE, PHYS_CHARGE, blocksparse_inputs, blocksparse_structure,
                       haar_unitary, heisenberg_mpo, sector_dims, tebd_inputs)


def test_sector_dims_config():
    d = sector_dims(2048, 15, 5.0)
    assert len(d) == 31 and int(d.sum()) == 2048 and d.min() >= 1
    assert np.all(d == d[::-1])                      # symmetric in q
    assert 150 <= d.max() <= 175 and d.argmax() == 15


def test_mpo_conserves_u1_charge():
    W = heisenberg_mpo()
    for wl in range(5):
        for wr in range(5):
            for s in range(2):
                for t in range(2):
                    if W[wl, wr, s, t] != 0:
                        assert PHYS_CHARGE[s] - PHYS_CHARGE[t] == MPO_CHANNEL_CHARGE[wl] - MPO_CHANNEL_CHARGE[wr]


def test_blocksparse_equals_dense_and_respects_charge():
    inp = blocksparse_inputs(total=64, seed=3, qmax=5, sigma=2.0)
    blocks, dense = blocksparse.bs_heff_apply(inp)
    dims = inp["dims"]
    off = np.concatenate([[0], np.cumsum(dims)[:-1]])
    # the dense result vanishes outside the allowed blocks (charge conservation)
    mask = np.zeros(dense.shape, dtype=bool)
    for (ia, s1, s2, ib) in blocksparse_structure(dims, inp["qmax"])["psi"]:
        mask[off[ia]:off[ia] + dims[ia], s1, s2, off[ib]:off[ib] + dims[ib]] = True
    assert np.max(np.abs(dense[~mask])) < 1e-12 * np.max(np.abs(dense))
    # the other contraction order (L first) on the same zero-filled tensors
    psiD = blocksparse.densify_psi({k: v.astype(float) for k, v in inp["psi"].items()}, dims)
    LD = blocksparse.densify_env({k: v.astype(float) for k, v in inp["L"].items()}, dims)
    RD = blocksparse.densify_env({k: v.astype(float) for k, v in inp["R"].items()}, dims)
    ref = heff.heff_apply(LD, inp["W"], RD, psiD, order="L")
    assert rel_frob_err(dense, ref) < 1e-13
    flops = blocksparse.bs_flops(inp)
    assert 0 < flops < heff.heff_flops(64)


def _brute_force_bs_heff(inp):
    """out and the multiply-add count of the block-sparse H_eff, by explicit loops.

    Works on the zero-filled (densified) tensors and reads the block structure
    from their nonzero pattern only (no block lists): stage 1 takes one
    multiply-add per pair psi[a',t1,t2,b'] != 0, R[b,wr,b'] != 0; stage 2 applies
    the 20 x 20 W.W matrix on every (a', b) pair where some U[a',:,:,b,:] != 0;
    stage 3 takes one multiply-add per L[a,wl,a'] != 0 and (a', b) pair carrying
    U, for every output element whose block is allowed (psi's pattern).
    """
    dims = inp["dims"]
    P = blocksparse.densify_psi({k: v.astype(float) for k, v in inp["psi"].items()}, dims)
    L = blocksparse.densify_env({k: v.astype(float) for k, v in inp["L"].items()}, dims)
    R = blocksparse.densify_env({k: v.astype(float) for k, v in inp["R"].items()}, dims)
    W = inp["W"]
    n, Dw, d = L.shape[0], W.shape[0], W.shape[2]
    U = np.zeros((n, d, d, n, Dw))
    mac1 = 0
    for ap, t1, t2, bp in zip(*np.nonzero(P)):
        for b in range(n):
            for wr in range(Dw):
                if R[b, wr, bp] != 0.0:
                    U[ap, t1, t2, b, wr] += P[ap, t1, t2, bp] * R[b, wr, bp]
                    mac1 += 1
    V = np.zeros((d, d, n, Dw, n))
    carries = np.zeros((n, n), dtype=bool)
    mac2 = 0
    for ap in range(n):
        for b in range(n):
            if not np.any(U[ap, :, :, b, :] != 0.0):
                continue
            carries[ap, b] = True
            for wl in range(Dw):
                for s1 in range(d):
                    for s2 in range(d):
                        acc = 0.0
                        for wr in range(Dw):
                            for t1 in range(d):
                                for t2 in range(d):
                                    ww = 0.0
                                    for wm in range(Dw):
                                        ww += W[wl, wm, s1, t1] * W[wm, wr, s2, t2]
                                    acc += ww * U[ap, t1, t2, b, wr]
                                    mac2 += 1
                        V[s1, s2, b, wl, ap] = acc
    out = np.zeros((n, d, d, n))
    mac3 = 0
    for a, s1, s2, b in zip(*np.nonzero(P)):
        acc = 0.0
        for wl in range(Dw):
            for ap in range(n):
                if L[a, wl, ap] != 0.0 and carries[ap, b]:
                    acc += L[a, wl, ap] * V[s1, s2, b, wl, ap]
                    mac3 += 1
        out[a, s1, s2, b] = acc
    return out, mac1, mac2, mac3


def _asymmetric_bs_inputs(dims, seed):
    """Block-sparse inputs with the given (not mirror-symmetric) sector dims, q = -qmax..qmax."""
    dims = np.asarray(dims, dtype=np.int64)
    qmax = (len(dims) - 1) // 2
    st = blocksparse_structure(dims, qmax)
    rng = np.random.default_rng(seed)
    draw = lambda k, j: rng.standard_normal((dims[k[0]], dims[k[j]])).astype(np.float32)
    return {"dims": dims, "qmax": qmax, "psi": {k: draw(k, 3) for k in st["psi"]},
            "L": {k: draw(k, 2) for k in st["L"]}, "R": {k: draw(k, 2) for k in st["R"]},
            "W": heisenberg_mpo(1.0)}


@pytest.mark.parametrize("case", ["gaussian", "asymmetric"])
def test_blocksparse_brute_force_sum_and_flop_count(case):
    if case == "gaussian":
        # 5 sectors (dims 1, 3, 4, 3, 1): the edge sectors leave some (a', b) pairs without U
        inp = blocksparse_inputs(total=12, seed=11, qmax=2, sigma=1.0)
        assert list(inp["dims"]) == [1, 3, 4, 3, 1]
    else:
        # no mirror symmetry, so a swapped operand dimension changes the count
        inp = _asymmetric_bs_inputs([2, 1, 4, 3, 1, 2, 1], seed=12)
    out_bf, mac1, mac2, mac3 = _brute_force_bs_heff(inp)
    _, dense = blocksparse.bs_heff_apply(inp)
    assert rel_frob_err(dense, out_bf) < 1e-13
    n = int(np.sum(inp["dims"]))
    assert mac1 > 0 and mac2 > 0 and mac3 > 0
    assert mac2 % 400 == 0 and mac2 // 400 < n * n        # not every (a', b) pair carries U
    assert blocksparse.bs_flops(inp) == 2.0 * (mac1 + mac2 + mac3)


def test_blocksparse_flop_count_config():
    inp = blocksparse_inputs(total=2048, seed=1)
    fl = blocksparse.bs_flops(inp)
    assert 1e9 < fl < 6.905e11 / 4


def test_tebd_identity_gate_and_unitarity():
    chis, A, B, G = tebd_inputs(4, seed=2, chi_lo=3, chi_hi=6)
    for a, b, g in zip(A, B, G):
        eye = np.eye(4).reshape(2, 2, 2, 2)
        th_id = tebd.theta(a, b, eye)
        ab = contract(a.astype(complex), "aic", b.astype(complex), "cjb", "aijb")
        assert rel_frob_err(th_id, np.transpose(ab, (0, 1, 2, 3))) < 1e-15
        th = tebd.theta(a, b, g)
        # unitary G preserves the Frobenius norm
        assert abs(np.linalg.norm(th) - np.linalg.norm(ab)) < 1e-5 * np.linalg.norm(ab)
        # brute-force sum on the (tiny) bond
        bf = contract_bruteforce(g.astype(complex), "stij", ab, "aijb", "astb")
        assert rel_frob_err(th, bf) < 1e-13


def test_tebd_3m_equals_4m():
    chis, A, B, G = tebd_inputs(3, seed=5, chi_lo=5, chi_hi=9)
    for a, b in zip(A, B):
        ref = contract(a.astype(complex), "aic", b.astype(complex), "cjb", "aijb")
        assert rel_frob_err(tebd.ab_3m(a, b), ref) < 1e-14


def test_tebd_gate_conventions_agree_for_symmetric_gate():
    rng = np.random.default_rng(4)
    U = haar_unitary(4, rng)
    S = U @ U.T                                      # complex symmetric unitary
    chis, A, B, _ = tebd_inputs(1, seed=6, chi_lo=4, chi_hi=4)
    g = S.reshape(2, 2, 2, 2)
    # paper convention sums u's first two indices; ours sums G's last two
    ours = tebd.theta(A[0], B[0], g)
    paper = tebd.theta_paper_convention(A[0], B[0], g)
    assert rel_frob_err(ours, paper) < 1e-13
    gu = U.reshape(2, 2, 2, 2)
    assert rel_frob_err(tebd.theta(A[0], B[0], gu), tebd.theta_paper_convention(A[0], B[0], gu)) > 1e-3


def test_haar_unitary_is_unitary():
    rng = np.random.default_rng(7)
    U = haar_unitary(4, rng)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(4), atol=1e-14)


def test_bf16_rounding_and_split():
    # exact bf16 values round to themselves; midpoints go to even
    x = np.array([1.0, 1.0078125, -2.5, 3.0e-3], dtype=np.float32)
    np.testing.assert_array_equal(precision.bf16_round(x[:3]), x[:3])
    one_plus_half_ulp = np.float32(1.0 + 2.0 ** -8)      # midpoint between 1 and 1+2^-7
    assert precision.bf16_round(np.array([one_plus_half_ulp]))[0] == 1.0
    three_halves_ulp = np.float32(1.0 + 3 * 2.0 ** -8)   # midpoint between 1+2^-7 and 1+2^-6
    assert precision.bf16_round(np.array([three_halves_ulp]))[0] == np.float32(1.0 + 2.0 ** -6)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(10000)
    hi, mid, lo = precision.split3(v)
    np.testing.assert_array_equal(hi.astype(np.float64) + mid + lo, v.astype(np.float32).astype(np.float64))
    for p in (hi, mid, lo):
        np.testing.assert_array_equal(precision.bf16_round(p), p)


def test_split_product_error_levels():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((64, 512))
    B = rng.standard_normal((512, 64))
    ref = A @ B
    e6 = rel_frob_err(precision.split_matmul(A, B, 6), ref)
    e3 = rel_frob_err(precision.split_matmul(A, B, 3), ref)
    assert e6 < 1e-7 < 1e-6 < e3 < 1e-4
