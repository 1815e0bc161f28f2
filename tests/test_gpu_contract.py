"""GPU parity of the TCI tensor calls and the generic contraction vs the oracle."""
import json
import os

import numpy as np
import pytest

from conftest import to_dev
from oracle.contract import contract as o_contract, rel_frob_err
from tci_synth import random_tensor

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))

PATTERNS = [
    ("ij", "jkl", "ikl", {"i": 33, "j": 17, "k": 2, "l": 29}),
    ("ijk", "kl", "ijl", {"i": 31, "j": 2, "k": 45, "l": 70}),
    ("ijk", "klm", "ijlm", {"i": 20, "j": 2, "k": 37, "l": 2, "m": 19}),
    ("ijkl", "lm", "ijkm", {"i": 9, "j": 2, "k": 2, "l": 65, "m": 33}),
    ("ijkl", "jkmn", "imnl", {"i": 40, "j": 2, "k": 2, "l": 41, "m": 2, "n": 2}),
    ("ijk", "kjl", "li", {"i": 3, "j": 4, "k": 2, "l": 5}),
    ("ijkl", "lmno", "ijkmno", {"i": 2, "j": 3, "k": 2, "l": 7, "m": 2, "n": 3, "o": 2}),
    ("ij", "ij", "", {"i": 130, "j": 77}),
    ("i", "j", "ji", {"i": 300, "j": 257}),
    ("abc", "cbd", "da", {"a": 200, "b": 5, "c": 300, "d": 260}),
]


@pytest.mark.parametrize("la,lb,lc,dims", PATTERNS)
@pytest.mark.parametrize("dtype", [np.float64, np.complex128, np.float32, np.complex64])
def test_contract_native_matches_oracle(ctx, tci, la, lb, lc, dims, dtype):
    A = random_tensor([dims[c] for c in la], 1, dtype)
    B = random_tensor([dims[c] for c in lb], 2, dtype)
    ref = o_contract(A.astype(np.complex128 if np.iscomplexobj(A) else np.float64), la,
                     B.astype(np.complex128 if np.iscomplexobj(B) else np.float64), lb, lc)
    out = tci.contract(ctx, to_dev(A), la, to_dev(B), lb, lc).cpu().numpy()
    tol = 1e-13 if dtype in (np.float64, np.complex128) else 2e-6
    assert out.shape == ref.shape
    assert rel_frob_err(out, ref) < tol


@pytest.mark.parametrize("la,lb,lc,dims", PATTERNS)
@pytest.mark.parametrize("prec,tol", [("split_bf16", 1e-6), ("split_bf16_3", 3e-5)])
def test_contract_split_bf16_matches_oracle(ctx, tci, la, lb, lc, dims, prec, tol):
    ctx.set_precision(prec)
    A = random_tensor([dims[c] for c in la], 3)
    B = random_tensor([dims[c] for c in lb], 4)
    ref = o_contract(A, la, B, lb, lc)
    out = tci.contract(ctx, to_dev(A), la, to_dev(B), lb, lc).cpu().numpy()
    assert rel_frob_err(out, ref) < tol


def test_contract_split_bf16_f32_operands(ctx, tci):
    ctx.set_precision("split_bf16")
    A = random_tensor([130, 300], 5, np.float32)
    B = random_tensor([300, 270], 6, np.float32)
    ref = o_contract(A.astype(np.float64), "ik", B.astype(np.float64), "kj", "ij")
    out = tci.contract(ctx, to_dev(A), "ik", to_dev(B), "kj", "ij").cpu().numpy()
    assert out.dtype == np.float32 and rel_frob_err(out, ref) < 1e-6


def test_paper_contract_example(ctx, tci):
    g = GOLD["contract_ijk_kjl_li"]
    A = random_tensor(g["shape_a"], 5, np.float32)
    B = random_tensor(g["shape_b"], 6, np.float32)
    ta, tb = ctx.wrap(to_dev(A)), ctx.wrap(to_dev(B))
    c1 = tci.contract_into(ctx, ta, g["labels_a_int"], tb, g["labels_b_int"], None, g["labels_c_int"])
    c2 = tci.contract_into(ctx, ta, g["labels_a"], tb, g["labels_b"], None, g["labels_c"])
    assert list(c1.shape) == g["shape_c"] == list(c2.shape)
    ref = o_contract(A.astype(float), "ijk", B.astype(float), "kjl", "li")
    assert rel_frob_err(c1.to_numpy(), ref) < 2e-6
    np.testing.assert_array_equal(c1.to_numpy(), c2.to_numpy())


def test_aliasing_output_and_lazy_transpose(ctx, tci):
    # iTEBD-style in-place update Theta = contract(Theta, "ijk", Lambda, "kl", "ijl")
    th = random_tensor([7, 2, 9], 7)
    lam = random_tensor([9, 9], 8)
    t = tci.allocate(ctx, [7, 2, 9])
    t.from_numpy(th)
    tl = tci.allocate(ctx, [9, 9])
    tl.from_numpy(lam)
    tci.contract_into(ctx, t, "ijk", tl, "kl", t, "ijl")
    assert rel_frob_err(t.to_numpy(), o_contract(th, "ijk", lam, "kl", "ijl")) < 1e-13
    # lazy in-place transpose is read in place by the next contraction
    t.transpose_([2, 0, 1])
    assert t.shape == (9, 7, 2)
    ref_t = np.transpose(o_contract(th, "ijk", lam, "kl", "ijl"), (2, 0, 1))
    np.testing.assert_array_equal(t.to_numpy(), ref_t)
    c = tci.contract_into(ctx, t, "lij", tl, "lm", None, "ijm")
    assert rel_frob_err(c.to_numpy(), o_contract(ref_t, "lij", lam, "lm", "ijm")) < 1e-13


def test_reshape_transpose_examples(ctx, tci):
    g = GOLD["reshape_342"]
    a = tci.allocate(ctx, g["shape"], zero=True)
    a.reshape_(g["new_shape"])
    assert list(a.shape) == g["new_shape"]
    b = a.reshape(g["second_new_shape"])
    assert list(b.shape) == g["second_new_shape"]
    s = GOLD["size_bytes_float_342"]
    f = tci.allocate(ctx, s["shape"], dtype=tci.F32)
    assert f.size() == s["size"] and f.size_bytes() == s["size_bytes"]
    g = GOLD["transpose_324"]
    x = random_tensor(g["shape"], 9)
    t = tci.allocate(ctx, g["shape"])
    t.from_numpy(x)
    e1 = x[tuple(g["elem_before"])]
    t.transpose_(g["new_order"])
    assert t.to_numpy()[tuple(g["elem_after"])] == e1
    u = t.transpose(g["second_order"])
    assert list(u.shape) == g["second_shape"]
    np.testing.assert_array_equal(u.to_numpy(), np.transpose(np.transpose(x, g["new_order"]), g["second_order"]))
    # reshape after a lazy transpose materialises in logical row-major order
    t.reshape_([2, 12])
    np.testing.assert_array_equal(t.to_numpy(), np.transpose(x, g["new_order"]).reshape(2, 12))


def test_norm_scale_close_linear_combine(ctx, tci):
    import torch
    n = GOLD["norm_eye3"]
    e = ctx.wrap(torch.eye(n["n"], dtype=torch.float64, device="cuda"))
    assert abs(e.norm() ** 2 - n["norm_squared"]) < 1e-15
    sc = GOLD["scale_eye3"]
    m = torch.eye(3, dtype=torch.float64, device="cuda")
    ctx.wrap(m).scale_(sc["s"])
    assert m[2, 2].item() == sc["elem_22"]
    cl = GOLD["close_eye3"]
    A = torch.eye(3, dtype=torch.float64, device="cuda")
    B = A.clone()
    B[tuple(cl["perturb_at"])] = cl["perturb"]
    assert not tci.close(ctx, A, B, cl["eps_false"])
    assert tci.close(ctx, A, B, cl["eps_true"])
    x = random_tensor([3, 4, 2], 1)
    tx = ctx.wrap(to_dev(x))
    old = tx.normalize_()
    assert abs(old - np.linalg.norm(x)) < 1e-12 and abs(tx.norm() - 1) < 1e-14
    xs = [random_tensor([3, 4, 2], s) for s in (1, 2, 3)]
    out = torch.empty(3, 4, 2, dtype=torch.float64, device="cuda")
    tci.linear_combine(ctx, [to_dev(v) for v in xs], [1.0, 2.0, 3.0], out)
    np.testing.assert_allclose(out.cpu().numpy(), xs[0] + 2 * xs[1] + 3 * xs[2], rtol=1e-14, atol=1e-14)


def test_error_codes(ctx, tci):
    import torch
    a = torch.zeros(3, 3, dtype=torch.float64, device="cuda")
    b = torch.zeros(3, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(tci.TciError) as ei:
        tci.contract(ctx, a, "ii", b, "ij", "j")
    assert ei.value.status_name == "TCI_ERR_LABEL"
    with pytest.raises(tci.TciError) as ei:
        tci.contract(ctx, a, "ij", b, "kl", "il")          # free bonds j, k missing from c
    assert ei.value.status_name == "TCI_ERR_UNSUPPORTED"
    with pytest.raises(tci.TciError) as ei:
        tci.contract(ctx, a, "ij", torch.zeros(4, 4, dtype=torch.float64, device="cuda"), "jk", "ik")
    assert ei.value.status_name == "TCI_ERR_LABEL"
    with pytest.raises(tci.TciError) as ei:
        tci.contract(ctx, a, "ij", b.float(), "jk", "ik")
    assert ei.value.status_name == "TCI_ERR_DTYPE"


def test_empty_and_degenerate(ctx, tci):
    import torch
    a = torch.zeros(0, 5, dtype=torch.float64, device="cuda")
    b = torch.ones(5, 3, dtype=torch.float64, device="cuda")
    out = tci.contract(ctx, a, "ik", b, "kj", "ij")
    assert tuple(out.shape) == (0, 3)
    a = torch.ones(4, 0, dtype=torch.float64, device="cuda")
    b = torch.ones(0, 3, dtype=torch.float64, device="cuda")
    out = tci.contract(ctx, a, "ik", b, "kj", "ij")
    assert torch.all(out == 0) and tuple(out.shape) == (4, 3)


BATCH_PATTERNS = [
    ("ij", "jk", "ijk", {"i": 33, "j": 17, "k": 29}),                    # batch bond j
    ("bij", "bjk", "bik", {"b": 70, "i": 31, "j": 45, "k": 19}),          # batched matrix product
    ("ibj", "jkb", "kbi", {"i": 9, "b": 130, "j": 65, "k": 2}),           # batch in the middle, permuted output
    ("ab", "ab", "ab", {"a": 300, "b": 257}),                             # elementwise product
    ("abc", "cbd", "bad", {"a": 20, "b": 3, "c": 40, "d": 26}),           # one batch, one summed
    ("aij", "ajk", "aik", {"a": 70000, "i": 2, "j": 3, "k": 2}),          # > 65535 batch slices
    ("ij", "ij", "i", {"i": 5, "j": 0}),                                  # summed bond of size 0: zeros
]


@pytest.mark.parametrize("la,lb,lc,dims", BATCH_PATTERNS)
@pytest.mark.parametrize("dtype", [np.float64, np.complex128, np.float32])
@pytest.mark.parametrize("prec", ["native", "split_bf16"])
def test_contract_batch_bonds_match_oracle(ctx, tci, la, lb, lc, dims, dtype, prec):
    """Labels in a, b and c: one product per batch slice (native arithmetic in every precision)."""
    ctx.set_precision(prec)
    try:
        A = random_tensor([dims[c] for c in la], 3, dtype)
        B = random_tensor([dims[c] for c in lb], 4, dtype)
        wide = np.complex128 if np.iscomplexobj(A) else np.float64
        ref = o_contract(A.astype(wide), la, B.astype(wide), lb, lc)
        out = tci.contract(ctx, to_dev(A), la, to_dev(B), lb, lc).cpu().numpy()
    finally:
        ctx.set_precision("native")
    assert out.shape == ref.shape
    if ref.size == 0 or not np.any(ref):
        assert np.all(out == 0)
        return
    if prec == "split_bf16" and dtype != np.complex128:
        tol = 3e-6                          # real slices run on the split-BF16 tensor cores
    else:
        tol = 1e-13 if dtype in (np.float64, np.complex128) else 2e-6
    assert rel_frob_err(out, ref) < tol


@pytest.mark.parametrize("la,lb,lc,shape", [("sab", "sAb", "aA", (3, 5, 4)),       # plain: Gram matrix
                                            ("zsa", "zsA", "zaA", (6, 2, 7)),      # batch bond z
                                            ("zsab", "zsAb", "zaA", (4, 2, 3, 5))])
def test_contract_one_tensor_as_both_operands(ctx, tci, la, lb, lc, shape):
    """The same handle passed as a and b: each operand keeps its own strides."""
    A = random_tensor(list(shape), 8)
    t = ctx.wrap(to_dev(A))
    out = tci.contract_into(ctx, t, la, t, lb, None, lc).to_numpy()
    np.testing.assert_allclose(out, o_contract(A, la, A, lb, lc), atol=1e-12)


@pytest.mark.parametrize("la,lb,lc,dims", [("zsab", "zsAb", "zaA", {"z": 3, "s": 2, "a": 20, "A": 20, "b": 3000}),
                                           ("ik", "jk", "ij", {"i": 33, "j": 70, "k": 20000}),
                                           ("kij", "kjl", "il", {"k": 7, "i": 5, "j": 2048, "l": 9})])
@pytest.mark.parametrize("dtype", [np.float64, np.complex128, np.float32])
def test_contract_split_k_matches_oracle(ctx, tci, la, lb, lc, dims, dtype):
    """Few output tiles and a long summed bond: the native GEMM splits K and adds the partials in order."""
    A = random_tensor([dims[c] for c in la], 5, dtype)
    B = random_tensor([dims[c] for c in lb], 6, dtype)
    wide = np.complex128 if np.iscomplexobj(A) else np.float64
    ref = o_contract(A.astype(wide), la, B.astype(wide), lb, lc)
    out = tci.contract(ctx, to_dev(A), la, to_dev(B), lb, lc).cpu().numpy()
    tol = 1e-13 if dtype in (np.float64, np.complex128) else 2e-6
    assert rel_frob_err(out, ref) < tol
