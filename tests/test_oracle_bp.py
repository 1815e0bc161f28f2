"""Pins of oracle/bp.py (App. B belief propagation on a TNS norm network)."""
import itertools

import numpy as np
import pytest

from oracle import bp as o_bp
from tci_synth import bp_tns_inputs, heavy_hex_graph

TREE = (7, [(0, 1), (0, 2), (0, 3), (1, 4), (1, 5), (3, 6)])


def full_state(n, edges, V):
    """psi[s_0 .. s_{n-1}]: the network contracted over every bond (einsum)."""
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    phys = [next(letters) for _ in range(n)]
    bond = {e: next(letters) for e in range(len(edges))}
    nb = o_bp.neighbours(n, edges)
    terms = []
    for i in range(n):
        sub = phys[i]
        for (w, m_in) in nb[i]:
            sub += bond[m_in // 2]
        terms.append(sub)
    return np.einsum(",".join(terms) + "->" + "".join(phys), *V)


def exact_density(psi, i):
    m = np.moveaxis(psi, i, 0).reshape(psi.shape[i], -1)
    rho = m @ m.T
    return rho / np.trace(rho)


def test_bp_is_exact_on_a_tree():
    n, edges = TREE
    V, M = bp_tns_inputs(n, edges, 3, seed=5)
    M, res = o_bp.bp(n, edges, V, M, 12)
    assert res[-1] < 1e-13                     # a tree converges in diameter + 1 iterations
    psi = full_state(n, edges, V)
    for i in range(n):
        np.testing.assert_allclose(o_bp.site_density(n, edges, V, M, i), exact_density(psi, i), atol=1e-12)


def test_message_equals_written_out_sum():
    rng = np.random.default_rng(1)
    V = rng.standard_normal((2, 2, 3, 2))      # site with three bonds of dims 2, 3, 2
    M0, M2 = rng.standard_normal((2, 2)), rng.standard_normal((2, 2))
    got = o_bp.message_update(V, [M0, None, M2], 1)
    ref = np.zeros((3, 3))
    for b, bp_ in itertools.product(range(3), range(3)):
        for s, a, a2, c, c2 in itertools.product(range(2), range(2), range(2), range(2), range(2)):
            ref[b, bp_] += V[s, a, b, c] * V[s, a2, bp_, c2] * M0[a, a2] * M2[c, c2]
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_product_state_is_exact_on_the_loopy_lattice():
    n, edges = heavy_hex_graph(3, 5)
    V, M = bp_tns_inputs(n, edges, 1, seed=2)
    M, res = o_bp.bp(n, edges, V, M, 3)
    for i in (0, 7, n - 1):
        v = V[i].reshape(-1)
        np.testing.assert_allclose(o_bp.site_density(n, edges, V, M, i), np.outer(v, v) / (v @ v), atol=1e-14)


def test_fixed_point_messages_are_psd_and_consistent():
    n, edges = heavy_hex_graph(2, 5)
    V, M = bp_tns_inputs(n, edges, 2, seed=3)
    M, res = o_bp.bp(n, edges, V, M, 200, tol=1e-12)
    assert res[-1] <= 1e-12
    for m in M:
        np.testing.assert_allclose(m, m.T, atol=1e-12)
        assert np.linalg.eigvalsh(m).min() > -1e-12
        assert abs(np.linalg.norm(m) - 1.0) < 1e-12
    M2, r2 = o_bp.bp_iteration(n, edges, V, M)
    assert r2 <= 2e-12


def test_heavy_hex_structure():
    n, edges = heavy_hex_graph(4, 9)
    deg = np.bincount(np.array(edges).ravel(), minlength=n)
    assert deg.max() == 3 and deg.min() >= 1
    assert np.all(deg[36:] == 2)                 # one inserted vertex per brick-wall bond
    assert len(set(edges)) == len(edges) == 2 * (n - 36)
