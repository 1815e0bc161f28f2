"""Pins for oracles O2/O3: MPO, exact environments and the two-site H_eff."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import heff
from oracle.contract import rel_frob_err
from tci_synth import dense_heff_inputs, heisenberg_mpo, random_tensor

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))

# Spin-1/2 operators built from the Pauli matrices, independently of tci_synth.
_PX = np.array([[0, 1], [1, 0]], dtype=float)
_PY_IM = np.array([[0, -1], [1, 0]], dtype=float)   # sigma_y = i * _PY_IM
_PZ = np.array([[1, 0], [0, -1]], dtype=float)
_SZ = _PZ / 2
_SP = (_PX - _PY_IM) / 2        # (sigma_x + i sigma_y)/2 = [[0,1],[0,0]]
_SM = (_PX + _PY_IM) / 2


def kron_heisenberg(n, J=1.0, sparse=True):
    """H = J sum_i [ (S+_i S-_{i+1} + S-_i S+_{i+1})/2 + Sz_i Sz_{i+1} ], open chain."""
    kron = sp.kron if sparse else np.kron
    eye = (lambda m: sp.identity(m, format="csr")) if sparse else np.eye

    def op2(A, B, i):
        return kron(kron(eye(2 ** i), kron(A, B)), eye(2 ** (n - i - 2)))

    H = None
    for i in range(n - 1):
        term = J * (0.5 * (op2(_SP, _SM, i) + op2(_SM, _SP, i)) + op2(_SZ, _SZ, i))
        H = term if H is None else H + term
    return H


def heff_from_envs(nl, nr):
    W = heisenberg_mpo(1.0)
    return heff.left_env(W, nl), W, heff.right_env(W, nr)


def test_mpo_chain_equals_kronecker():
    W = heisenberg_mpo(1.0)
    for n in (2, 3, 4, 6):
        np.testing.assert_allclose(heff.mpo_chain_matrix(W, n), kron_heisenberg(n, sparse=False),
                                   atol=1e-14)


def test_two_site_spectrum():
    L, W, R = heff_from_envs(0, 0)
    H = heff.heff_matrix_loops(L, W, R)
    ev = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(ev, GOLD["heisenberg_obc_ground"]["two_site_spectrum"], atol=1e-14)


@pytest.mark.parametrize("n,e0", [(3, -1.0), (4, -(3 + 2 * np.sqrt(3)) / 4)])
def test_small_chain_closed_forms(n, e0):
    H = kron_heisenberg(n, sparse=False)
    assert abs(np.linalg.eigvalsh(H)[0] - e0) < 1e-13


@pytest.mark.parametrize("order", ["L", "R"])
def test_heff_orders_match_explicit_matrix(order):
    # chi = 3 on the left, 2 on the right: explicit loop matrix times psi.
    psi, L, R, W = dense_heff_inputs(3, seed=11, chi_r=2)
    Hm = heff.heff_matrix_loops(L, W, R)
    ref = (Hm @ psi.ravel()).reshape(psi.shape)
    out = heff.heff_apply(L, W, R, psi, order=order)
    assert rel_frob_err(out, ref) < 1e-14


@pytest.mark.parametrize("chi,chi_r", [(8, 8), (16, 12), (33, 17)])
def test_heff_contraction_order_independence(chi, chi_r):
    psi, L, R, W = dense_heff_inputs(chi, seed=3, chi_r=chi_r)
    a = heff.heff_apply(L, W, R, psi, order="L")
    b = heff.heff_apply(L, W, R, psi, order="R")
    assert rel_frob_err(a, b) < 1e-13


def test_heff_rows_sampling_matches_full():
    psi, L, R, W = dense_heff_inputs(24, seed=5)
    full = heff.heff_apply(L, W, R, psi)
    rows = [0, 7, 23]
    assert rel_frob_err(heff.heff_rows(L, W, R, psi, rows), full[rows]) < 1e-13


def test_identity_mpo_returns_psi():
    chi = 6
    psi = random_tensor([chi, 2, 2, chi], 9)
    W = np.eye(2).reshape(1, 1, 2, 2)
    E = np.eye(chi).reshape(chi, 1, chi)
    out = heff.heff_apply(E, W, E, psi)
    np.testing.assert_array_equal(out, psi)


@pytest.mark.parametrize("nl,nr", [(4, 4), (3, 5)])
def test_exact_envs_give_full_hamiltonian_10_sites(nl, nr):
    L, W, R = heff_from_envs(nl, nr)
    n = nl + nr + 2
    Hk = kron_heisenberg(n, sparse=False)
    # H_eff(env) == H elementwise, checked by acting on the identity columns in blocks
    dim = 2 ** n
    X = np.eye(dim)[:, ::7]
    cols = [heff.heff_apply(L, W, R, X[:, k].reshape(L.shape[0], 2, 2, R.shape[0])).ravel()
            for k in range(X.shape[1])]
    np.testing.assert_allclose(np.stack(cols, 1), Hk @ X, atol=1e-13)


def test_exact_envs_12_sites_action():
    L, W, R = heff_from_envs(5, 5)
    assert L.shape == (32, 5, 32) and R.shape == (32, 5, 32)
    Hk = kron_heisenberg(12)
    for seed in (1, 2):
        x = random_tensor([32, 2, 2, 32], seed)
        np.testing.assert_allclose(heff.heff_apply(L, W, R, x).ravel(), Hk @ x.ravel(), atol=1e-12)


def test_symmetrised_envs_make_heff_symmetric():
    psi, L, R, W = dense_heff_inputs(12, seed=21)
    x = random_tensor(psi.shape, 1)
    y = random_tensor(psi.shape, 2)
    lhs = np.vdot(x, heff.heff_apply(L, W, R, y))
    rhs = np.vdot(heff.heff_apply(L, W, R, x), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-12
    # without symmetrisation the matrix is not symmetric (guards the sigma map)
    psi2, L2, R2, W2 = dense_heff_inputs(12, seed=21, symmetrise=False)
    lhs2 = np.vdot(x, heff.heff_apply(L2, W2, R2, y))
    rhs2 = np.vdot(heff.heff_apply(L2, W2, R2, x), y)
    assert abs(lhs2 - rhs2) > 1e-6 * abs(lhs2)


def test_ed_ground_energy_10_sites():
    Hk = kron_heisenberg(10)
    e0 = spla.eigsh(Hk, k=1, which="SA", tol=1e-13)[0][0]
    Hd = kron_heisenberg(10, sparse=False)
    assert abs(np.linalg.eigvalsh(Hd)[0] - e0) < 1e-10
    assert -4.3 < e0 < -4.2


def test_flop_count_formula():
    chi = 2048
    assert heff.heff_flops(chi) == 4 * chi ** 3 * 4 * 5 + 2 * chi ** 2 * 16 * 25
    assert abs(heff.heff_flops(2048) - 6.905e11) / 6.905e11 < 1e-3


@pytest.mark.parametrize("chi,chi_r,Dw,d", [(2, 3, 2, 2), (3, 2, 3, 3)])
def test_complex_heff_matches_explicit_matrix(chi, chi_r, Dw, d):
    """Complex L, W, R, psi: both contraction orders equal the loop-built dense matrix (no conjugation)."""
    from tci_synth import complex_heff_inputs
    psi, L, R, W = complex_heff_inputs(chi, 7, chi_r, Dw, d)
    H = heff.heff_matrix_loops(L, W, R)
    ref = (H @ psi.ravel()).reshape(psi.shape)
    for order in ("L", "R"):
        np.testing.assert_allclose(heff.heff_apply(L, W, R, psi, order), ref, atol=1e-12)


@pytest.mark.parametrize("order", ["L", "R"])
def test_two_different_site_mpos_match_explicit_matrix(order):
    """W on the left site and W2 on the right one (a non-uniform MPO): both orders equal the loops."""
    rng = np.random.default_rng(12)
    L, R = rng.standard_normal((3, 5, 3)), rng.standard_normal((2, 5, 2))
    W, W2 = rng.standard_normal((5, 5, 2, 2)), rng.standard_normal((5, 5, 2, 2))
    psi = rng.standard_normal((3, 2, 2, 2))
    ref = (heff.heff_matrix_loops(L, W, R, W2) @ psi.ravel()).reshape(psi.shape)
    np.testing.assert_allclose(heff.heff_apply(L, W, R, psi, order, W2=W2), ref, atol=1e-12)
    assert np.abs(heff.heff_apply(L, W, R, psi, order) - ref).max() > 1e-3     # W2 matters
