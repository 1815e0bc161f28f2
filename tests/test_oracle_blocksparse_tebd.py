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
    # block-by-block recomputation with only the allowed blocks, by brute-force sums
    psiD = blocksparse.densify_psi({k: v.astype(float) for k, v in inp["psi"].items()}, dims)
    LD = blocksparse.densify_env({k: v.astype(float) for k, v in inp["L"].items()}, dims)
    RD = blocksparse.densify_env({k: v.astype(float) for k, v in inp["R"].items()}, dims)
    ref = heff.heff_apply(LD, inp["W"], RD, psiD, order="L")
    assert rel_frob_err(dense, ref) < 1e-13
    flops = blocksparse.bs_flops(inp)
    assert 0 < flops < heff.heff_flops(64)


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
