"""Pins of oracle/dmrg.py: exact diagonalisation of open Heisenberg chains and the environment identities."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import dmrg as o_dmrg
from oracle import heff as o_heff
from tci_synth import heisenberg_mpo


def ed_ground(n):
    from test_oracle_heff import kron_heisenberg
    H = kron_heisenberg(n)
    if n <= 10:
        return float(np.linalg.eigvalsh(H.toarray() if hasattr(H, "toarray") else H)[0])
    return float(spla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0])


def test_two_site_singlet():
    e, _ = o_dmrg.dmrg(heisenberg_mpo(), 2, 4, 2)
    assert abs(e[-1] + 0.75) < 1e-13


@pytest.mark.parametrize("n", [4, 6, 8, 10, 12])
def test_dmrg_matches_ed_without_truncation(n):
    """chi_max >= 2^(n/2): no truncation, the sweep converges to the exact ground energy."""
    e, errs = o_dmrg.dmrg(heisenberg_mpo(), n, 2 ** (n // 2), 4)
    assert abs(e[-1] - ed_ground(n)) < 1e-10 * abs(ed_ground(n))
    assert max(errs) < 1e-20


def test_truncated_dmrg_is_variational_and_close():
    n = 14
    e, errs = o_dmrg.dmrg(heisenberg_mpo(), n, 16, 4)
    e0 = ed_ground(n)
    assert e[-1] >= e0 - 1e-10                # variational: above the exact energy
    assert e[-1] - e0 < 1e-4 * abs(e0)        # and close at chi = 16
    assert max(errs) > 0.0


def test_environment_updates_match_exact_environments():
    """Updates with the identity-like computational basis reproduce the exact environments."""
    W = heisenberg_mpo()
    Lk = np.zeros((1, 5, 1)); Lk[0, 4, 0] = 1.0
    Rk = np.zeros((1, 5, 1)); Rk[0, 0, 0] = 1.0
    for k in range(3):
        chi = Lk.shape[0]
        A = np.eye(chi * 2).reshape(chi, 2, chi * 2)          # isometry onto the full basis
        Lk = o_dmrg.update_left(Lk, A, W)
        chi_r = Rk.shape[0]
        B = np.eye(2 * chi_r).reshape(2 * chi_r, 2, chi_r)
        Rk = o_dmrg.update_right(Rk, B, W)
    np.testing.assert_array_equal(Lk, o_heff.left_env(W, 3))
    np.testing.assert_array_equal(Rk, o_heff.right_env(W, 3))


def test_long_chain_bulk_energy_density():
    """Open chains of 32 and 64 sites at chi_max 32 (4 sweeps): in the bulk energy per site
    (E_64 - E_32) / 32 the boundary energy cancels, and it approaches the infinite chain's
    1/4 - ln 2 (Hulthen's Bethe-ansatz value).  What remains is the conformal 1/N term of the open
    chain, -pi^2 v c / (24 N) with v = pi/2, c = 1, which leaves pi^2 / (48 * 64 * 32) = 1.0e-4 in
    the difference, plus the truncation at chi 32: tolerance 3e-4.  The energy per site of the
    64-site chain alone is further off (the boundary energy over 64 sites), within 1e-2."""
    e_inf = 0.25 - np.log(2.0)
    e32, _ = o_dmrg.dmrg(heisenberg_mpo(), 32, 32, 4)
    e64, _ = o_dmrg.dmrg(heisenberg_mpo(), 64, 32, 4)
    bulk = (e64[-1] - e32[-1]) / 32
    assert abs(bulk - e_inf) < 3e-4, bulk
    assert 0.0 < bulk - e_inf < 3e-4          # the 1/N term raises the finite-chain difference
    assert abs(e64[-1] / 64 - e_inf) < 1e-2
    assert e64[-1] / 64 > e_inf               # open boundaries cost energy
