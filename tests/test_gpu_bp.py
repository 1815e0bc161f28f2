"""Device belief propagation (App. B) against the oracle's message iteration."""
import numpy as np
import pytest

from oracle import bp as o_bp
from tci_synth import bp_tns_inputs, heavy_hex_graph

pytestmark = pytest.mark.gpu

TREE = (7, [(0, 1), (0, 2), (0, 3), (1, 4), (1, 5), (3, 6)])


def _compare(tci, ctx, n, edges, V, M, niters, tol=0.0, atol=1e-12):
    got, res = tci.bp(ctx, n, edges, V, M, niters, tol)
    ref, rres = o_bp.bp(n, edges, V, M, niters, tol)
    assert len(res) == len(rres)
    np.testing.assert_allclose(res, rres, rtol=1e-9, atol=1e-12)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r, atol=atol)
    return got, res


@pytest.mark.parametrize("niters", [1, 2, 8])
def test_bp_tree_matches_oracle(ctx, tci, niters):
    n, edges = TREE
    V, M = bp_tns_inputs(n, edges, 3, seed=5)
    _compare(tci, ctx, n, edges, V, M, niters)


@pytest.mark.parametrize("rows,cols,chi", [(3, 5, 4), (2, 4, 7), (4, 9, 2)])
def test_bp_heavy_hex_matches_oracle(ctx, tci, rows, cols, chi):
    n, edges = heavy_hex_graph(rows, cols)
    V, M = bp_tns_inputs(n, edges, chi, seed=11)
    _compare(tci, ctx, n, edges, V, M, 6)


def test_bp_mixed_bond_dimensions_and_leaves(ctx, tci):
    # a ring with a tail; bond dimensions differ per edge; vertex 5 is a leaf
    n, edges = 6, [(0, 1), (1, 2), (2, 3), (0, 3), (3, 4), (4, 5)]
    dims = {e: d for e, d in zip(edges, [2, 3, 4, 5, 3, 2])}
    rng = np.random.default_rng(4)
    nb = o_bp.neighbours(n, edges)
    V = []
    for i in range(n):
        shape = [2] + [dims[tuple(sorted((i, w)))] for (w, _) in nb[i]]
        V.append(rng.standard_normal(shape))
    M = []
    for (u, v) in edges:
        d = dims[(u, v)]
        M += [np.eye(d) / np.sqrt(d), np.eye(d) / np.sqrt(d)]
    _compare(tci, ctx, n, edges, V, M, 10)


def test_bp_stops_at_tolerance(ctx, tci):
    n, edges = TREE
    V, M = bp_tns_inputs(n, edges, 2, seed=1)
    got, res = _compare(tci, ctx, n, edges, V, M, 50, tol=1e-12)
    assert len(res) < 50 and res[-1] <= 1e-12


def test_bp_rejects_bad_input(ctx, tci):
    n, edges = TREE
    V, M = bp_tns_inputs(n, edges, 2, seed=1)
    with pytest.raises(RuntimeError):
        tci.bp(ctx, n, edges + [(0, 1)], V, M + M[:2], 2)          # repeated edge
    with pytest.raises(RuntimeError):
        tci.bp(ctx, n, edges, V, [np.eye(3)] + M[1:], 2)            # message shape
    with pytest.raises(RuntimeError):
        tci.bp(ctx, n, [(0, 9)] + edges[1:], V, M, 2)               # vertex out of range


def test_bp_isolated_site_and_zero_iterations(ctx, tci):
    """A vertex without bonds carries no messages; zero iterations return the start messages."""
    n, edges = 5, [(0, 1), (1, 2), (2, 3)]          # vertex 4 is isolated
    V, M = bp_tns_inputs(n, edges, 3, seed=9)
    _compare(tci, ctx, n, edges, V, M, 4)
    got, res = tci.bp(ctx, n, edges, V, M, 0)
    assert res == [] and all(np.array_equal(g, m) for g, m in zip(got, M))


@pytest.mark.parametrize("chi", [4, 16])
def test_bp_split_precision_close_to_oracle(ctx, tci, chi):
    """Under the split-BF16 context precision the batched contractions run on the tensor cores."""
    n, edges = heavy_hex_graph(3, 5)
    V, M = bp_tns_inputs(n, edges, chi, seed=13)
    ctx.set_precision("split_bf16")
    try:
        got, res = tci.bp(ctx, n, edges, V, M, 5)
    finally:
        ctx.set_precision("native")
    ref, rres = o_bp.bp(n, edges, V, M, 5)
    np.testing.assert_allclose(res, rres, rtol=1e-4, atol=1e-6)
    for g, r in zip(got, ref):
        assert np.linalg.norm(g - r) < 1e-5
