"""Pins of oracle/linalg.py (TCI svd / trunc_svd): the paper's examples, exact identities, crafted spectra."""
import json
import os

import numpy as np
import pytest

from oracle import linalg as o
from tci_synth import random_tensor

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def test_svd_paper_example_shapes_and_identities():
    g = GOLD["svd_example"]
    a = random_tensor(g["shape"], 1)
    u, s, vt = o.svd(a, g["k"])
    assert list(u.shape) == g["u_shape"] and list(s.shape) == g["s_shape"] and list(vt.shape) == g["vt_shape"]
    m = a.reshape(12, 12)
    um, vm = u.reshape(12, 12), vt.reshape(12, 12)
    np.testing.assert_allclose(um @ np.diag(s) @ vm, m, atol=1e-13)      # reconstruction
    np.testing.assert_allclose(um.T @ um, np.eye(12), atol=1e-13)       # orthonormal columns
    np.testing.assert_allclose(vm @ vm.T, np.eye(12), atol=1e-13)
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    # singular values are the square roots of the eigenvalues of A'^T A'
    np.testing.assert_allclose(np.sort(s ** 2), np.linalg.eigvalsh(m.T @ m), rtol=1e-12, atol=1e-12)


def test_trunc_svd_paper_example():
    g = GOLD["trunc_svd_example"]
    a = random_tensor(g["shape"], 2)
    u, s, vt, err = o.trunc_svd(a, g["k"], g["chi_min"], g["chi_max"], g["target_trunc_err"], g["s_min"])
    assert err != 0.0
    assert g["chi_min"] <= s.shape[0] <= g["chi_max"]


def _with_spectrum(s, seed=3, shape=(6, 8)):
    rng = np.random.default_rng(seed)
    q1, _ = np.linalg.qr(rng.standard_normal((shape[0], shape[0])))
    q2, _ = np.linalg.qr(rng.standard_normal((shape[1], shape[1])))
    m = np.zeros(shape)
    m[:len(s), :len(s)] = np.diag(s)
    return q1 @ m @ q2.T


def test_trunc_rules_on_a_known_spectrum():
    s = np.array([4.0, 2.0, 1.0, 0.5, 1e-3, 1e-9])
    a = _with_spectrum(s)
    tot = float(np.sum(s ** 2))
    # (1) fixed chi_max, s_min: keep the 3 largest
    u, sk, vt, err = o.trunc_svd(a, 1, 1, 3, 0.0, 0.0)
    assert sk.shape == (3,) and abs(err - (0.25 + 1e-6 + 1e-18) / tot) < 1e-15
    # (a) s_min removes the two smallest even with a large chi_max
    assert o.trunc_count(s, 1, 10, 0.0, 1e-2) == 4
    # (b) fewer than chi_min remain after (a): keep those
    assert o.trunc_count(s, 5, 10, 0.0, 0.6) == 3
    # (c) grow from chi_min until eps <= target
    assert o.trunc_count(s, 1, 10, (1.0 + 0.25 + 1e-6 + 1e-18) / tot, 0.0) == 2
    assert o.trunc_count(s, 1, 10, 0.3 / tot, 0.0) == 3
    assert o.trunc_count(s, 1, 10, 0.05 / tot, 0.0) == 4
    # chi_max caps (c)
    assert o.trunc_count(s, 1, 2, 0.0, 0.0) == 2
    np.testing.assert_allclose(sk, s[:3], rtol=1e-13)


def test_svd_rejects_bad_row_count():
    with pytest.raises(ValueError):
        o.svd(np.zeros((2, 3)), 2)
