"""Pins of oracle/itebd.py (the App. A iteration): exact TFIM energies, limits and the gate."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import itebd as o
from tci_synth import itebd_initial_state, tfim_bond_hamiltonian


def test_gate_is_the_matrix_exponential():
    h = tfim_bond_hamiltonian(1.0, 0.7)
    np.testing.assert_allclose(o.gate(h, 0.03).reshape(4, 4), sla.expm(-0.03 * h), atol=1e-15)


def test_exact_energy_closed_forms():
    assert abs(o.tfim_exact_energy(1.0, 1.0) + 4.0 / np.pi) < 1e-12        # critical point: -4/pi
    assert abs(o.tfim_exact_energy(1.0, 0.0) + 1.0) < 1e-12                # classical Ising
    assert abs(o.tfim_exact_energy(0.0, 2.5) + 2.5) < 1e-12                # free spins in a field


def test_classical_limit_converges_exactly():
    gam, lam = itebd_initial_state(4, 7)
    e, _, lm = o.itebd(tfim_bond_hamiltonian(1.0, 0.0), 0.05, gam, lam, 4, 400)
    assert abs(e[-1] + 1.0) < 1e-12


@pytest.mark.parametrize("g,chi,dt,n,tol", [(0.5, 16, 0.01, 2000, 1e-6), (1.0, 16, 0.01, 2000, 2e-4),
                                            (3.0, 8, 0.02, 1000, 2e-4)])
def test_energy_approaches_the_exact_solution(g, chi, dt, n, tol):
    gam, lam = itebd_initial_state(chi, 7)
    e, _, lm = o.itebd(tfim_bond_hamiltonian(1.0, g), dt, gam, lam, chi, n)
    assert abs(e[-1] - o.tfim_exact_energy(1.0, g)) < tol
    assert abs(np.linalg.norm(lm[(n - 1) % 2]) - 1.0) < 1e-12      # Lambda_A normalised
