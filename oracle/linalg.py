"""TCI ``svd`` and ``trunc_svd`` (paper App. C.2, Tensor linear algebra), written out.

Test infrastructure only.  Definitions followed:

* ``svd(a, k)``: matricise a by grouping its first k bonds into the row
  index and the rest into the column index (A' is I x J), factor
  A' = U S V^dagger with s_0 >= ... >= s_{kappa-1} >= 0, kappa = min(I, J), and
  fold back: u [d_0..d_{k-1}, kappa], s [kappa], v_dag [kappa, d_k..d_{r-1}].
  The factorisation itself is the library routine (``numpy.linalg.svd``).
* ``trunc_svd``: the truncation error of keeping chi values is
  eps(chi) = sum_{i >= chi} s_i^2 / sum_i s_i^2; the retained count follows the
  paper's three rules in order: (a) discard every s_i < s_min; (b) keep at
  least chi_min values, or all that remain after (a) if fewer; (c) add values
  in descending order until eps <= target_trunc_err or chi = chi_max.
  Reading where the rules are silent: chi_max caps the count (chi_min is
  lowered to chi_max when it exceeds it) and at least one value is kept when
  any s_i >= s_min.
"""
from __future__ import annotations

import numpy as np


def matricise(a, k):
    a = np.asarray(a)
    if not 1 <= k < a.ndim:
        raise ValueError("num_of_bds_as_row must satisfy 1 <= k < order")
    I = int(np.prod(a.shape[:k], dtype=np.int64))
    J = int(np.prod(a.shape[k:], dtype=np.int64))
    return a.reshape(I, J), a.shape[:k], a.shape[k:]


def svd(a, k):
    m, rs, cs = matricise(a, k)
    u, s, vt = np.linalg.svd(m, full_matrices=False)
    kappa = s.shape[0]
    return u.reshape(tuple(rs) + (kappa,)), s, vt.reshape((kappa,) + tuple(cs))


def trunc_error(s, chi):
    s = np.asarray(s, dtype=np.float64)
    tot = float(np.sum(s * s))
    return float(np.sum(s[chi:] ** 2)) / tot if tot > 0 else 0.0


def trunc_count(s, chi_min, chi_max, target_trunc_err, s_min):
    """Number of singular values kept (s in non-increasing order)."""
    s = np.asarray(s, dtype=np.float64)
    remain = int(np.sum(s >= s_min))                  # rule (a)
    chi_min = min(chi_min, chi_max)
    if remain <= chi_min:                             # rule (b)
        return remain
    chi = chi_min
    while chi < min(chi_max, remain) and trunc_error(s, chi) > target_trunc_err:   # rule (c)
        chi += 1
    return chi


def trunc_svd(a, k, chi_min, chi_max, target_trunc_err, s_min):
    """(u, s, v_dag, trunc_err) with the kept count from ``trunc_count``."""
    u, s, vt = svd(a, k)
    chi = trunc_count(s, chi_min, chi_max, target_trunc_err, s_min)
    return u[..., :chi], s[:chi], vt[:chi], trunc_error(s, chi)
