"""O1: label-based Einstein contraction (TCI core function ``contract``).

Definition (paper Sec. II.B.2, Eq. for C_IJ): tensors A and B share the bond
set S; I are A's other bonds, J are B's other bonds;
    C_{IJ} = sum_S A_{IS} B_{SJ}.
Label semantics (paper App. C.2, ``tci::contract``): a label present in both
operands and absent from the output is summed; the output's label list fixes
the free bonds and their order; an empty output label list gives a scalar;
repeating a label inside one operand is prohibited.

``contract`` follows the three-step recipe the paper gives for tensor
linear-algebra operations (Sec. II.B.2): matricise A to [I, S] and B to
[S, J], multiply (numpy matmul is the library primitive), refold to the
output's bond order.  ``contract_bruteforce`` is the sum written out
element by element and exists to pin ``contract``.

Readings where the paper is silent:
* a label in both operands *and* in the output (a batch bond) is read as
  "for every value of that label, contract the slices": C_{IJB} =
  sum_S A_{ISB} B_{SJB}, the same definition applied slice by slice;
* a label in one operand that is absent from the output (an implicit partial
  sum) is not covered by the specification -> ``UnsupportedLabels``.
"""
from __future__ import annotations

import itertools

import numpy as np


class LabelError(ValueError):
    """Repeated label within one operand, rank mismatch, or dimension mismatch."""


class UnsupportedLabels(ValueError):
    """Label pattern outside the TCI ``contract`` specification."""


def _as_list(labels):
    if isinstance(labels, str):
        return list(labels)
    return list(labels)


def classify(shape_a, la, shape_b, lb, lc):
    """Return (I, S, J, Bt, dims) label groups after validating the label lists.

    I: free bonds of a, J: free bonds of b, S: summed bonds (in a and b, not
    in c), Bt: batch bonds (in a, b and c); orders follow a (I, S, Bt) and b (J).
    """
    la, lb, lc = _as_list(la), _as_list(lb), _as_list(lc)
    if len(la) != len(shape_a) or len(lb) != len(shape_b):
        raise LabelError("label count differs from tensor order")
    for lab in (la, lb, lc):
        if len(set(lab)) != len(lab):
            raise LabelError("a label repeats within one operand")
    dims = {}
    for lab, shp in ((la, shape_a), (lb, shape_b)):
        for l, d in zip(lab, shp):
            if l in dims and dims[l] != d:
                raise LabelError(f"bond dimension mismatch for label {l!r}")
            dims[l] = int(d)
    S = [l for l in la if l in lb and l not in lc]
    I = [l for l in la if l not in lb]
    J = [l for l in lb if l not in la]
    Bt = [l for l in la if l in lb and l in lc]
    if sorted(map(str, lc)) != sorted(map(str, I + J + Bt)):
        raise UnsupportedLabels("output labels must be exactly the free and batch bonds of a and b")
    return I, S, J, Bt, dims


def contract(A, la, B, lb, lc):
    """C = contract(A, la, B, lb, lc); float64/complex128 in, same kind out."""
    A = np.asarray(A)
    B = np.asarray(B)
    la, lb, lc = _as_list(la), _as_list(lb), _as_list(lc)
    I, S, J, Bt, dims = classify(A.shape, la, B.shape, lb, lc)
    size = lambda labels: int(np.prod([dims[l] for l in labels], dtype=np.int64))
    nI, nS, nJ, nB = size(I), size(S), size(J), size(Bt)
    # matricise every batch slice: A -> [Bt][I, S], B -> [Bt][S, J]
    Am = np.transpose(A, [la.index(l) for l in Bt + I + S]).reshape(nB, nI, nS)
    Bm = np.transpose(B, [lb.index(l) for l in Bt + S + J]).reshape(nB, nS, nJ)
    Cm = np.empty((nB, nI, nJ), dtype=np.result_type(A.dtype, B.dtype))
    for t in range(nB):                   # one matrix product per batch slice
        Cm[t] = Am[t] @ Bm[t]
    C = Cm.reshape([dims[l] for l in Bt + I + J])
    perm = [(Bt + I + J).index(l) for l in lc]
    return np.transpose(C, perm).copy()


def contract_bruteforce(A, la, B, lb, lc):
    """The same contraction as an explicit sum over every coordinate (tiny sizes only)."""
    A = np.asarray(A)
    B = np.asarray(B)
    la, lb, lc = _as_list(la), _as_list(lb), _as_list(lc)
    I, S, J, Bt, dims = classify(A.shape, la, B.shape, lb, lc)
    out_shape = tuple(dims[l] for l in lc)
    dtype = np.result_type(A.dtype, B.dtype)
    C = np.zeros(out_shape, dtype=dtype)
    for oc in itertools.product(*[range(d) for d in out_shape]):
        coord = dict(zip(lc, oc))
        acc = dtype.type(0)
        for sc in itertools.product(*[range(dims[l]) for l in S]):
            coord.update(zip(S, sc))
            acc += A[tuple(coord[l] for l in la)] * B[tuple(coord[l] for l in lb)]
        C[oc] = acc
    return C


def frob_norm(A) -> float:
    """Frobenius norm (paper App. C.2, ``tci::norm``, Eq. frob_norm)."""
    A = np.asarray(A)
    return float(np.sqrt(np.sum(np.abs(A) ** 2)))


def rel_frob_err(x, ref) -> float:
    """||x - ref||_F / ||ref||_F."""
    return frob_norm(np.asarray(x) - np.asarray(ref)) / frob_norm(ref)


def close(A, B, eps) -> bool:
    """TCI ``close``: shapes equal and max |A - B| <= eps (paper App. C.2)."""
    A = np.asarray(A)
    B = np.asarray(B)
    if A.shape != B.shape:
        return False
    return bool(np.max(np.abs(A - B)) <= eps) if A.size else True
