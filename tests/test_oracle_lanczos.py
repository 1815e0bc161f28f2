"""Pins for oracle O4 (Lanczos, Sturm bisection, inverse iteration)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import heff, lanczos
from tci_synth import dense_heff_inputs, heisenberg_mpo, random_tensor
from test_oracle_heff import kron_heisenberg


def test_sturm_bisection_matches_eigvalsh():
    rng = np.random.default_rng(0)
    for m in (1, 2, 5, 20, 40):
        a = rng.standard_normal(m)
        b = rng.standard_normal(max(m - 1, 0))
        T = lanczos.tridiag_matrix(a, b)
        ref = np.linalg.eigvalsh(T)[0]
        assert abs(lanczos.lowest_eigenvalue_bisect(a, b) - ref) < 1e-12 * max(1, abs(ref))
        # Sturm counts against the full spectrum
        ev = np.linalg.eigvalsh(T)
        for x in np.linspace(ev[0] - 1, ev[-1] + 1, 9):
            assert lanczos.sturm_count(a, b, x) == int(np.sum(ev < x))


def test_tridiag_eigvec():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(12)
    b = rng.standard_normal(11)
    T = lanczos.tridiag_matrix(a, b)
    th = lanczos.lowest_eigenvalue_bisect(a, b)
    y = lanczos.tridiag_eigvec(a, b, th)
    assert np.linalg.norm(T @ y - th * y) < 1e-10
    assert abs(np.linalg.norm(y) - 1) < 1e-14


def test_two_site_singlet_exact():
    W = heisenberg_mpo(1.0)
    L = heff.left_env(W, 0)
    R = heff.right_env(W, 0)
    v0 = random_tensor([1, 2, 2, 1], 3)
    res = lanczos.lanczos(lambda v: heff.heff_apply(L, W, R, v.reshape(1, 2, 2, 1)), v0, 10)
    assert abs(res["theta"] - (-0.75)) < 1e-14


@pytest.mark.parametrize("nl,nr", [(4, 4), (3, 5)])
def test_lanczos_matches_ed_10_sites(nl, nr):
    W = heisenberg_mpo(1.0)
    L = heff.left_env(W, nl)
    R = heff.right_env(W, nr)
    shape = (L.shape[0], 2, 2, R.shape[0])
    e0 = spla.eigsh(kron_heisenberg(nl + nr + 2), k=1, which="SA", tol=1e-14)[0][0]
    v0 = random_tensor(shape, 4)
    res = lanczos.lanczos(lambda v: heff.heff_apply(L, W, R, v.reshape(shape)), v0, 80)
    assert abs(res["theta"] - e0) < 1e-10
    # the Ritz vector is an eigenvector
    x = res["x"]
    Hx = heff.heff_apply(L, W, R, x.reshape(shape)).ravel()
    assert np.linalg.norm(Hx - res["theta"] * x) < 1e-6


def test_lanczos_12_sites_config1_shape():
    W = heisenberg_mpo(1.0)
    L = heff.left_env(W, 5)
    R = heff.right_env(W, 5)
    shape = (32, 2, 2, 32)
    e0 = spla.eigsh(kron_heisenberg(12), k=1, which="SA", tol=1e-14)[0][0]
    res = lanczos.lanczos(lambda v: heff.heff_apply(L, W, R, v.reshape(shape)), random_tensor(shape, 5), 120)
    assert abs(res["theta"] - e0) < 1e-10


def test_lanczos_basis_orthonormal_and_tridiagonal():
    psi, L, R, W = dense_heff_inputs(6, seed=8)
    shape = psi.shape
    mv = lambda v: heff.heff_apply(L, W, R, v.reshape(shape))
    res = lanczos.lanczos(mv, psi, 20)
    # rebuild the basis by the same recurrence and check V^T H V == T
    a, b = res["alpha"], res["beta"]
    T = lanczos.tridiag_matrix(a, b[: len(a) - 1])
    ev = np.linalg.eigvalsh(T)
    assert abs(ev[0] - res["theta"]) < 1e-12 * max(1, abs(ev[0]))
    # Ritz value is an upper bound of the true ground energy (Courant-Fischer)
    Hm = np.stack([mv(e.reshape(shape)).ravel() for e in np.eye(np.prod(shape))], 1)
    assert res["theta"] >= np.linalg.eigvalsh(0.5 * (Hm + Hm.T))[0] - 1e-10


def test_lanczos_deterministic():
    psi, L, R, W = dense_heff_inputs(8, seed=9)
    mv = lambda v: heff.heff_apply(L, W, R, v.reshape(psi.shape))
    r1 = lanczos.lanczos(mv, psi, 20)
    r2 = lanczos.lanczos(mv, psi, 20)
    assert r1["theta"] == r2["theta"]


def test_sturm_count_with_an_exact_zero_pivot():
    """x equal to alpha_0 makes the first pivot exactly zero; the count must stay right.

    T = [[-1/4, 1/2], [1/2, -1/4]] has eigenvalues -3/4 and 1/4: one lies below -1/4.
    """
    from oracle.lanczos import lowest_eigenvalue_bisect, sturm_count
    alpha, beta = [-0.25, -0.25], [0.5]
    assert sturm_count(alpha, beta, -0.25) == 1
    assert abs(lowest_eigenvalue_bisect(alpha, beta) + 0.75) < 1e-15


def test_real_form_lanczos_finds_hermitian_ground_energy():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    H = 0.5 * (a + a.conj().T)
    r = lanczos.lanczos_real_form(lambda v: H @ v, rng.standard_normal(40) + 0j, 80)
    assert abs(r["theta"] - np.linalg.eigvalsh(H)[0]) < 1e-10
    x = r["x"]
    assert np.linalg.norm(H @ x - r["theta"] * x) < 1e-8 and abs(np.linalg.norm(x) - 1.0) < 1e-12


def test_hermitian_heff_and_its_ground_energy():
    from tci_synth import hermitian_heff_inputs
    psi, L, R, W = hermitian_heff_inputs(3, 4, 2)
    H = heff.heff_matrix_loops(L, W, R)
    np.testing.assert_allclose(H, H.conj().T, atol=1e-12)                  # the symmetrisation works
    r = lanczos.lanczos_real_form(lambda v: heff.heff_apply(L, W, R, v), psi, 2 * H.shape[0])
    assert abs(r["theta"] - np.linalg.eigvalsh(H)[0]) < 1e-9
