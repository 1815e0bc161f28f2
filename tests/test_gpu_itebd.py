"""Device iTEBD (App. A) against the oracle's iteration and the exact TFIM ground energy."""
import numpy as np
import pytest

from oracle import itebd as o_itebd
from tci_synth import itebd_initial_state, tfim_bond_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("g,chi,dt,n,tol", [(0.5, 8, 0.02, 600, 1e-5), (1.0, 16, 0.01, 2000, 2e-4),
                                            (3.0, 8, 0.02, 600, 2e-4)])
def test_itebd_matches_oracle_and_exact(ctx, tci, g, chi, dt, n, tol):
    h = tfim_bond_hamiltonian(1.0, g)
    gam, lam = itebd_initial_state(chi, 7)
    e, terr, G, L = tci.itebd(ctx, h, dt, gam, lam, chi, n)
    re, rG, rL = o_itebd.itebd(h, dt, gam, lam, chi, n)
    # gauge-invariant: Theta' norms of the first iterations agree to rounding
    np.testing.assert_allclose(e[:20], re[:20], rtol=0, atol=1e-10)
    assert abs(e[-1] - re[-1]) < 1e-8
    exact = o_itebd.tfim_exact_energy(1.0, g)
    assert abs(e[-1] - exact) < tol, (e[-1], exact)      # Trotter error O(dt^2) and truncation
    # Schmidt spectra (gauge-invariant) of the last bond agree; Lambda_A is normalised
    last = (n - 1) % 2
    assert L[last].shape == rL[last].shape
    np.testing.assert_allclose(L[last], rL[last], atol=1e-7)
    assert abs(np.linalg.norm(L[last]) - 1.0) < 1e-12
    assert all(t >= 0.0 for t in terr)
    assert G[last].shape[1] == 2 and G[last].shape[2] == L[last].shape[0]


def test_itebd_classical_limit(ctx, tci):
    gam, lam = itebd_initial_state(4, 3)
    e, _, _, L = tci.itebd(ctx, tfim_bond_hamiltonian(1.0, 0.0), 0.05, gam, lam, 4, 300)
    assert abs(e[-1] + 1.0) < 1e-12


def test_itebd_rejects_bad_cell(ctx, tci):
    gam, lam = itebd_initial_state(4, 3)
    with pytest.raises(RuntimeError):
        tci.itebd(ctx, tfim_bond_hamiltonian(), 0.01, gam, [lam[0], lam[1][:3]], 4, 5)
    with pytest.raises(RuntimeError):
        tci.itebd(ctx, tfim_bond_hamiltonian(), -0.01, gam, lam, 4, 5)


def test_itebd_bond_dimension_one(ctx, tci):
    """chi = 1 (product states): the device iteration equals the oracle's, energies stay above the exact one."""
    h = tfim_bond_hamiltonian(1.0, 0.8)
    gam, lam = itebd_initial_state(1, 4)
    e, _, G, L = tci.itebd(ctx, h, 0.02, gam, lam, 1, 200)
    re, _, _ = o_itebd.itebd(h, 0.02, gam, lam, 1, 200)
    np.testing.assert_allclose(e, re, rtol=0, atol=1e-10)
    assert L[1].shape == (1,) and abs(abs(L[1][0]) - 1.0) < 1e-12
