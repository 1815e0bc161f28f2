"""GPU Lanczos (FP64 vector arithmetic) vs the oracle and exact diagonalisation."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from conftest import to_dev
from oracle import heff as o_heff, lanczos as o_lanczos
from tci_synth import dense_heff_inputs, heisenberg_mpo, random_tensor

pytestmark = pytest.mark.gpu


def gpu_lanczos(tci, ctx, L, W, R, psi0, m, precision="native"):
    import torch
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision=precision)
    x = torch.empty(psi0.shape, dtype=torch.float64, device="cuda")
    res = plan.lanczos(to_dev(psi0), m, True, x)
    res["x"] = x.cpu().numpy()
    return res


def test_two_site_singlet(ctx, tci):
    W = heisenberg_mpo()
    L, R = o_heff.left_env(W, 0), o_heff.right_env(W, 0)
    r = gpu_lanczos(tci, ctx, L, W, R, random_tensor([1, 2, 2, 1], 3), 10)
    assert abs(r["theta"] + 0.75) < 1e-14
    assert r["steps"] <= 4      # breakdown: the Krylov space is at most 4-dimensional


@pytest.mark.parametrize("nl,nr", [(4, 4), (5, 5)])
def test_ed_through_gpu_lanczos(ctx, tci, nl, nr):
    from test_oracle_heff import kron_heisenberg
    W = heisenberg_mpo()
    L, R = o_heff.left_env(W, nl), o_heff.right_env(W, nr)
    e0 = spla.eigsh(kron_heisenberg(nl + nr + 2), k=1, which="SA", tol=1e-14)[0][0]
    r = gpu_lanczos(tci, ctx, L, W, R, random_tensor([L.shape[0], 2, 2, R.shape[0]], 4), 120)
    assert abs(r["theta"] - e0) < 1e-10


def test_lanczos_chi32_matches_oracle(ctx, tci):
    psi, L, R, W = dense_heff_inputs(32, seed=20251223)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 20)
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    assert r["steps"] == o["steps"] == 20
    np.testing.assert_allclose(r["alpha"], o["alpha"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(r["beta"], o["beta"], rtol=1e-10, atol=1e-10)
    assert abs(r["theta"] - o["theta"]) < 1e-10 * abs(o["theta"])
    assert np.linalg.norm(r["x"].ravel() - o["x"]) < 1e-8


def test_lanczos_chi1024_ritz_value(ctx, tci):
    psi, L, R, W = dense_heff_inputs(1024, seed=20251223)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 20)
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    assert abs(r["theta"] - o["theta"]) < 1e-10 * abs(o["theta"])


def test_lanczos_split_bf16_ritz_close(ctx, tci):
    psi, L, R, W = dense_heff_inputs(256, seed=7)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 20, precision="split_bf16")
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    assert abs(r["theta"] - o["theta"]) < 1e-6 * abs(o["theta"])
