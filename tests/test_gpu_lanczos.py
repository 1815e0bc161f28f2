"""GPU Lanczos (FP64 and double-float vector arithmetic) vs the oracle and exact diagonalisation."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from conftest import to_dev
from oracle import heff as o_heff, lanczos as o_lanczos
from tci_synth import dense_heff_inputs, heisenberg_mpo, random_tensor

pytestmark = pytest.mark.gpu


ARITH = ["f64", "df32"]


def gpu_lanczos(tci, ctx, L, W, R, psi0, m, precision="native", arith="auto", reorth=True, gs="dgks"):
    import torch
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision=precision)
    plan.set_lanczos_arith(arith)
    plan.set_gram_schmidt(gs)
    x = torch.empty(psi0.shape, dtype=torch.float64, device="cuda")
    res = plan.lanczos(to_dev(psi0), m, reorth, x)
    res["x"] = x.cpu().numpy()
    return res


@pytest.mark.parametrize("arith", ARITH)
def test_two_site_singlet(ctx, tci, arith):
    W = heisenberg_mpo()
    L, R = o_heff.left_env(W, 0), o_heff.right_env(W, 0)
    r = gpu_lanczos(tci, ctx, L, W, R, random_tensor([1, 2, 2, 1], 3), 10, arith=arith)
    assert abs(r["theta"] + 0.75) < 1e-14
    assert r["steps"] <= 4      # breakdown: the Krylov space is at most 4-dimensional


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("nl,nr", [(4, 4), (5, 5)])
def test_ed_through_gpu_lanczos(ctx, tci, nl, nr, arith):
    from test_oracle_heff import kron_heisenberg
    W = heisenberg_mpo()
    L, R = o_heff.left_env(W, nl), o_heff.right_env(W, nr)
    e0 = spla.eigsh(kron_heisenberg(nl + nr + 2), k=1, which="SA", tol=1e-14)[0][0]
    # 120 steps: the double-float basis exceeds one fused pass (24 vectors)
    r = gpu_lanczos(tci, ctx, L, W, R, random_tensor([L.shape[0], 2, 2, R.shape[0]], 4), 120, arith=arith)
    assert abs(r["theta"] - e0) < 1e-10


@pytest.mark.parametrize("gs", ["dgks", "twice"])
@pytest.mark.parametrize("arith", ARITH)
def test_lanczos_chi32_matches_oracle(ctx, tci, arith, gs):
    psi, L, R, W = dense_heff_inputs(32, seed=20251223)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 20, arith=arith, gs=gs)
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    assert r["steps"] == o["steps"] == 20
    np.testing.assert_allclose(r["alpha"], o["alpha"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(r["beta"], o["beta"], rtol=1e-10, atol=1e-10)
    assert abs(r["theta"] - o["theta"]) < 1e-10 * abs(o["theta"])
    assert np.linalg.norm(r["x"].ravel() - o["x"]) < 1e-8


@pytest.mark.parametrize("arith", ARITH)
def test_lanczos_chi1024_ritz_value(ctx, tci, arith):
    psi, L, R, W = dense_heff_inputs(1024, seed=20251223)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 20, arith=arith)
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    assert abs(r["theta"] - o["theta"]) < 1e-10 * abs(o["theta"])


def test_lanczos_split_bf16_ritz_close(ctx, tci):
    psi, L, R, W = dense_heff_inputs(256, seed=7)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 20, precision="split_bf16")
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    assert abs(r["theta"] - o["theta"]) < 1e-6 * abs(o["theta"])


@pytest.mark.parametrize("arith", ARITH)
def test_lanczos_without_reorth_matches_oracle(ctx, tci, arith):
    """Plain three-term recurrence (reorth off): 8 steps, before orthogonality is lost."""
    psi, L, R, W = dense_heff_inputs(24, seed=5)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 8, arith=arith, reorth=False)
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 8, reorth=False)
    np.testing.assert_allclose(r["alpha"], o["alpha"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(r["beta"], o["beta"], rtol=1e-10, atol=1e-10)
    assert abs(r["theta"] - o["theta"]) < 1e-10 * abs(o["theta"])


def test_lanczos_split_bf16_df_vs_f64_vectors(ctx, tci):
    """Split-BF16 plan, ragged chi (Kp padding): both vector arithmetics against the FP64 oracle."""
    psi, L, R, W = dense_heff_inputs(75, seed=11, chi_r=61)
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    for arith in ARITH:
        r = gpu_lanczos(tci, ctx, L, W, R, psi, 20, precision="split_bf16", arith=arith)
        assert abs(r["theta"] - o["theta"]) < 1e-6 * abs(o["theta"]), arith
        assert np.linalg.norm(np.abs(r["x"].ravel()) - np.abs(o["x"])) < 1e-4, arith
