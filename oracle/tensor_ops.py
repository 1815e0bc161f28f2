"""TCI construction and elementwise functions (paper App. C.2), written out.

Test infrastructure only (see the package docstring).  Each function is the
definition the paper states for it:

* ``eye`` (Tensor construction): the N x N identity, ones on the main
  diagonal and zeros elsewhere;
* ``fill`` (Tensor construction): every element equal to the given value;
* ``cplx_conj`` (Tensor manipulation): elementwise complex conjugation, no
  change for real tensors;
* ``to_cplx`` (Tensor manipulation): real elements embedded with zero
  imaginary parts; complex input copied;
* ``diag`` (Tensor linear algebra): a first-order tensor becomes the square
  matrix with it on the main diagonal; a second-order tensor gives its main
  diagonal of length min(d0, d1); other orders are an error.

Element-by-element loops (no numpy helpers such as ``np.eye``/``np.diag``),
so the pins in ``tests/test_oracle_tensor_ops.py`` can compare against those
library routines independently.
"""
from __future__ import annotations

import numpy as np


def eye(n: int, dtype=np.float64) -> np.ndarray:
    out = np.zeros((n, n), dtype=dtype)
    for i in range(n):
        out[i, i] = 1
    return out


def fill(shape, value, dtype=np.float64) -> np.ndarray:
    out = np.empty(tuple(shape), dtype=dtype)
    flat = out.reshape(-1)
    for i in range(flat.size):
        flat[i] = value
    return out


def cplx_conj(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a)
    if not np.iscomplexobj(a):
        return a.copy()
    out = np.empty_like(a)
    for idx in np.ndindex(a.shape):
        z = a[idx]
        out[idx] = complex(z.real, -z.imag)
    return out


def to_cplx(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return a.copy()
    out = np.empty(a.shape, dtype=np.complex64 if a.dtype == np.float32 else np.complex128)
    for idx in np.ndindex(a.shape):
        out[idx] = complex(a[idx], 0.0)
    return out


def diag(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a)
    if a.ndim == 1:
        n = a.shape[0]
        out = np.zeros((n, n), dtype=a.dtype)
        for i in range(n):
            out[i, i] = a[i]
        return out
    if a.ndim == 2:
        m = min(a.shape)
        out = np.empty((m,), dtype=a.dtype)
        for i in range(m):
            out[i] = a[i, i]
        return out
    raise ValueError("diag: input must be first- or second-order")
