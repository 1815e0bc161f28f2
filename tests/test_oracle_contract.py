"""Pins for oracle O1 (label contraction) against brute force and the paper's examples."""
import json
import os

import numpy as np
import pytest

from oracle.contract import (LabelError, UnsupportedLabels, close, contract, contract_bruteforce,
                             frob_norm)
from tci_synth import random_tensor

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))

# Contraction patterns that appear in the paper's iTEBD listing (App. A) and
# basic-usage example (Sec. III), plus the App. C.2 contract example.
PATTERNS = [
    ("ij", "jkl", "ikl", {"i": 3, "j": 4, "k": 2, "l": 3}),
    ("ijk", "kl", "ijl", {"i": 3, "j": 2, "k": 4, "l": 3}),
    ("ijk", "klm", "ijlm", {"i": 2, "j": 3, "k": 4, "l": 2, "m": 3}),
    ("ijkl", "lm", "ijkm", {"i": 2, "j": 3, "k": 2, "l": 4, "m": 3}),
    ("ijkl", "jkmn", "imnl", {"i": 3, "j": 2, "k": 2, "l": 3, "m": 2, "n": 2}),
    ("ijk", "kjl", "li", {"i": 3, "j": 4, "k": 2, "l": 5}),
    ("ijkl", "lmno", "ijkmno", {"i": 2, "j": 2, "k": 2, "l": 3, "m": 2, "n": 1, "o": 2}),
    ("ij", "ij", "", {"i": 3, "j": 4}),                   # full contraction -> scalar
    ("i", "j", "ij", {"i": 3, "j": 4}),                   # outer product
    ("ijk", "jk", "i", {"i": 5, "j": 3, "k": 2}),
]


@pytest.mark.parametrize("la,lb,lc,dims", PATTERNS)
@pytest.mark.parametrize("dtype", [np.float64, np.complex128])
def test_contract_matches_bruteforce(la, lb, lc, dims, dtype):
    A = random_tensor([dims[c] for c in la], 1, dtype)
    B = random_tensor([dims[c] for c in lb], 2, dtype)
    C = contract(A, la, B, lb, lc)
    Cb = contract_bruteforce(A, la, B, lb, lc)
    assert C.shape == tuple(dims[c] for c in lc)
    np.testing.assert_allclose(C, Cb, rtol=1e-13, atol=1e-13)


def test_contract_matches_hand_loop_gemm():
    # C[i,l] = sum_j A[i,j] B[j,l] written as explicit Python loops.
    A = random_tensor([4, 5], 3)
    B = random_tensor([5, 3], 4)
    C = contract(A, "ij", B, "jl", "il")
    for i in range(4):
        for l in range(3):
            s = 0.0
            for j in range(5):
                s += A[i, j] * B[j, l]
            assert abs(C[i, l] - s) < 1e-13


def test_paper_contract_example_shape():
    g = GOLD["contract_ijk_kjl_li"]
    A = random_tensor(g["shape_a"], 5)
    B = random_tensor(g["shape_b"], 6)
    C1 = contract(A, g["labels_a_int"], B, g["labels_b_int"], g["labels_c_int"])
    C2 = contract(A, g["labels_a"], B, g["labels_b"], g["labels_c"])
    assert list(C1.shape) == g["shape_c"] == list(C2.shape)
    np.testing.assert_allclose(C1, C2, rtol=0, atol=0)
    np.testing.assert_allclose(C2, contract_bruteforce(A, "ijk", B, "kjl", "li"), rtol=1e-13)


def test_identity_contraction():
    A = random_tensor([4, 3, 5], 7)
    eye = np.eye(5)
    np.testing.assert_array_equal(contract(A, "ijk", eye, "kl", "ijl"), A)
    eye4 = np.eye(4)
    np.testing.assert_array_equal(contract(eye4, "ai", A, "ijk", "ajk"), A)


def test_label_errors():
    A = random_tensor([3, 3], 1)
    B = random_tensor([3, 4], 2)
    with pytest.raises(LabelError):
        contract(A, "ii", B, "ij", "j")            # repeated label in one operand
    with pytest.raises(LabelError):
        contract(A, "ij", random_tensor([4, 4], 3), "jk", "ik")   # dim mismatch
    with pytest.raises(UnsupportedLabels):
        contract(A, "ij", B, "kl", "il")           # free bonds j, k dropped
    with pytest.raises(UnsupportedLabels):
        contract(A, "ij", B, "jk", "k")            # free bond i of a missing from c


@pytest.mark.parametrize("la,lb,lc,shapes", [
    ("ij", "jk", "ijk", ([3, 4], [4, 5])),                   # batch bond j (Hadamard along j, outer in i, k)
    ("bij", "bjk", "bik", ([4, 3, 5], [4, 5, 2])),           # batched matrix product
    ("ibj", "jkb", "kbi", ([3, 4, 2], [2, 5, 4])),           # batch bond in the middle, permuted output
    ("ab", "ab", "ab", ([3, 4], [3, 4])),                    # elementwise product (all bonds batch)
    ("abc", "cbd", "bad", ([2, 3, 4], [4, 3, 5])),           # one batch, one summed, permuted
])
def test_batch_bonds_match_bruteforce_and_einsum(la, lb, lc, shapes):
    A = random_tensor(shapes[0], 11) + 1j * random_tensor(shapes[0], 12)
    B = random_tensor(shapes[1], 13)
    ref = contract_bruteforce(A, la, B, lb, lc)
    np.testing.assert_allclose(contract(A, la, B, lb, lc), ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(np.einsum(f"{la},{lb}->{lc}", A, B), ref, rtol=1e-13, atol=1e-13)


def test_norm_and_close_examples():
    g = GOLD["norm_eye3"]
    assert abs(frob_norm(np.eye(g["n"])) ** 2 - g["norm_squared"]) < 1e-15
    c = GOLD["close_eye3"]
    A = np.eye(c["n"])
    B = A.copy()
    B[tuple(c["perturb_at"])] = c["perturb"]
    assert not close(A, B, c["eps_false"])
    assert close(A, B, c["eps_true"])
