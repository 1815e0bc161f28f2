"""Pins of oracle/tensor_ops.py: the paper's App. C.2 examples and library routines."""
import json
import os

import numpy as np
import pytest

from oracle import tensor_ops as o

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def test_eye_paper_example_and_numpy():
    g = GOLD["eye_3"]
    e = o.eye(g["n"])
    for idx, v in g["elems"]:
        assert e[tuple(idx)] == v
    np.testing.assert_array_equal(e, np.eye(5)[:3, :3])
    assert o.eye(0).shape == (0, 0)


def test_fill_paper_example():
    g = GOLD["fill_324"]
    a = o.fill(g["shape"], g["value"])
    assert a.shape == tuple(g["shape"])
    for idx, v in g["elems"]:
        assert a[tuple(idx)] == v
    assert np.all(a == g["value"])
    z = o.fill([2, 3], 1 - 2j, dtype=np.complex128)
    assert np.all(z == 1 - 2j)


def test_diag_paper_roundtrip_and_numpy():
    g = GOLD["diag_roundtrip_eye3"]
    a = o.eye(g["n"])
    d1 = o.diag(a)
    assert d1.ndim == g["order_after_first"]
    np.testing.assert_array_equal(o.diag(d1), a)
    rng = np.random.default_rng(3)
    r = rng.standard_normal((4, 6))
    np.testing.assert_array_equal(o.diag(r), np.diag(r))            # min(d0, d1) = 4
    v = rng.standard_normal(5)
    np.testing.assert_array_equal(o.diag(v), np.diag(v))
    with pytest.raises(ValueError):
        o.diag(np.zeros((2, 2, 2)))


def test_cplx_conj_and_to_cplx():
    g = GOLD["cplx_conj_elem"]
    rng = np.random.default_rng(4)
    a = rng.standard_normal(g["shape"]) + 1j * rng.standard_normal(g["shape"])
    c = o.cplx_conj(a)
    assert c[tuple(g["index"])] == np.conj(a[tuple(g["index"])])
    np.testing.assert_array_equal(c, np.conjugate(a))
    r = rng.standard_normal((3, 2))
    np.testing.assert_array_equal(o.cplx_conj(r), r)                  # real: unchanged (a copy)
    z = o.to_cplx(r.astype(np.float32))
    assert z.dtype == np.complex64 and np.all(z.imag == 0) and np.all(z.real == r.astype(np.float32))
    assert o.to_cplx(a) is not a and np.array_equal(o.to_cplx(a), a)
