"""GPU parity of the H_eff matvec (FP64 and split-BF16 paths) vs the oracle."""
import numpy as np
import pytest

from conftest import to_dev
from oracle import heff as o_heff
from oracle.contract import rel_frob_err
from tci_synth import dense_heff_inputs, heisenberg_mpo, random_tensor

pytestmark = pytest.mark.gpu


def run_heff(tci, ctx, L, W, R, psi, precision):
    import torch
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision=precision)
    out = torch.empty(psi.shape, dtype=torch.float64, device="cuda")
    plan.apply(to_dev(psi), out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), plan


@pytest.mark.parametrize("chi,chi_r", [(32, 32), (33, 17), (1, 1), (7, 130), (200, 64)])
def test_heff_fp64_matches_oracle(ctx, tci, chi, chi_r):
    psi, L, R, W = dense_heff_inputs(chi, seed=20251223, chi_r=chi_r)
    out, _ = run_heff(tci, ctx, L, W, R, psi, "native")
    ref = o_heff.heff_apply(L, W, R, psi)
    assert rel_frob_err(out, ref) < 1e-12


@pytest.mark.parametrize("chi,chi_r", [(32, 32), (33, 17), (130, 70), (300, 257)])
def test_heff_split_bf16_matches_oracle(ctx, tci, chi, chi_r):
    psi, L, R, W = dense_heff_inputs(chi, seed=1, chi_r=chi_r)
    out, _ = run_heff(tci, ctx, L, W, R, psi, "split_bf16")
    ref = o_heff.heff_apply(L, W, R, psi)
    assert rel_frob_err(out, ref) < 1e-6


def test_heff_split3_variant(ctx, tci):
    psi, L, R, W = dense_heff_inputs(96, seed=2)
    out, _ = run_heff(tci, ctx, L, W, R, psi, "split_bf16_3")
    assert rel_frob_err(out, o_heff.heff_apply(L, W, R, psi)) < 3e-5


def test_identity_mpo_fp64_returns_psi(ctx, tci):
    # Dw must be 5 for this build: embed the identity in channel 0 only
    chi = 24
    W = np.zeros((5, 5, 2, 2))
    W[0, 0] = np.eye(2)
    E = np.zeros((chi, 5, chi))
    E[:, 0, :] = np.eye(chi)
    psi = random_tensor([chi, 2, 2, chi], 4)
    out, _ = run_heff(tci, ctx, E, W, E, psi, "native")
    np.testing.assert_array_equal(out, psi)


@pytest.mark.parametrize("nl,nr", [(4, 4), (3, 5), (5, 5)])
def test_exact_envs_equal_full_hamiltonian(ctx, tci, nl, nr):
    from test_oracle_heff import kron_heisenberg
    W = heisenberg_mpo()
    L, R = o_heff.left_env(W, nl), o_heff.right_env(W, nr)
    psi = random_tensor([L.shape[0], 2, 2, R.shape[0]], 6)
    out, _ = run_heff(tci, ctx, L, W, R, psi, "native")
    ref = (kron_heisenberg(nl + nr + 2) @ psi.ravel()).reshape(psi.shape)
    assert rel_frob_err(out, ref) < 1e-13


def test_heff_fp64_chi1024_sampled_rows(ctx, tci):
    psi, L, R, W = dense_heff_inputs(1024, seed=20251223)
    out, plan = run_heff(tci, ctx, L, W, R, psi, "native")
    rows = [0, 1, 511, 777, 1023]
    ref = o_heff.heff_rows(L, W, R, psi, rows)
    assert rel_frob_err(out[rows], ref) < 1e-12
    assert plan.flops == o_heff.heff_flops(1024)


def test_heff_split_bf16_chi2048_full(ctx, tci):
    psi, L, R, W = dense_heff_inputs(2048, seed=20251223)
    out, plan = run_heff(tci, ctx, L, W, R, psi, "split_bf16")
    ref = o_heff.heff_apply(L, W, R, psi)        # full FP64 matvec (BLAS steps)
    err = rel_frob_err(out, ref)
    assert err < 1e-6, err


@pytest.mark.parametrize("chi,chi_r,prec", [(64, 64, "split_bf16"), (300, 257, "split_bf16"), (264, 40, "split_bf16"),
                                            (40, 33, "native")])
def test_apply_host_matches_device(ctx, tci, chi, chi_r, prec):
    """Host-buffer matvec (copies overlapped with compute in chunks of rows for chi >= 256) == device matvec."""
    psi, L, R, W = dense_heff_inputs(chi, seed=3, chi_r=chi_r)
    out, plan = run_heff(tci, ctx, L, W, R, psi, prec)
    host_out = np.full_like(psi, np.nan)
    plan.apply_host(np.ascontiguousarray(psi), host_out)
    np.testing.assert_array_equal(host_out, out)
    host_out2 = np.full_like(psi, np.nan)
    plan.apply_host(np.ascontiguousarray(psi), host_out2)      # repeated call reuses the staging buffers
    np.testing.assert_array_equal(host_out2, out)


@pytest.mark.parametrize("ww_na", [2, 4])
@pytest.mark.parametrize("chi,chi_r", [(33, 17), (130, 70), (64, 40)])
def test_heff_split_ww_variants(ctx, tci, chi, chi_r, ww_na):
    """Both W.W kernel variants (a' per thread 2 / 4), with ragged a' tails and unaligned rows."""
    import torch
    psi, L, R, W = dense_heff_inputs(chi, seed=9, chi_r=chi_r)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="split_bf16")
    c = plan.get_config()
    plan.set_config(c[0], c[1], c[2], ww_na)
    assert plan.get_config()[3] == ww_na
    dpsi = to_dev(psi)
    out = torch.full_like(dpsi, float("nan"))
    plan.apply(dpsi, out)
    torch.cuda.synchronize()
    assert rel_frob_err(out.cpu().numpy(), o_heff.heff_apply(L, W, R, psi)) < 1e-6


@pytest.mark.parametrize("prec,tol", [("native", 1e-12), ("split_bf16", 1e-6)])
def test_two_site_mpos_match_oracle(ctx, tci, prec, tol):
    """Different MPO tensors on the two sites (tci_heff_plan_create2) against the oracle."""
    import torch
    psi, L, R, W = dense_heff_inputs(40, seed=5, chi_r=33)
    W2 = random_tensor([5, 5, 2, 2], 6)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision=prec, W2=to_dev(W2))
    out = torch.full(psi.shape, float("nan"), dtype=torch.float64, device="cuda")
    plan.apply(to_dev(psi), out)
    torch.cuda.synchronize()
    assert rel_frob_err(out.cpu().numpy(), o_heff.heff_apply(L, W, R, psi, W2=W2)) < tol


@pytest.mark.parametrize("prec", ["native", "split_bf16"])
def test_plan_reload_equals_new_plan(ctx, tci, prec):
    """tci_heff_plan_reload: new environments (and a new MPO) in an existing plan give the same
    matvec and Lanczos results as a plan created from them, also after graph replays."""
    import torch
    psi, L1, R1, W = dense_heff_inputs(40, seed=3, chi_r=33)
    _, L2, R2, _ = dense_heff_inputs(40, seed=4, chi_r=33)
    W2 = random_tensor([5, 5, 2, 2], 8)
    plan = tci.HeffPlan(ctx, to_dev(L1), to_dev(W), to_dev(R1), precision=prec)
    dpsi = to_dev(psi)
    x = torch.empty_like(dpsi)
    for _ in range(3):                      # eager, captured, replayed
        plan.lanczos(dpsi, 12, True, x)
    for (L, R, Wn) in ((L2, R2, W), (L1, R1, W2)):
        plan.reload(to_dev(L), to_dev(Wn), to_dev(R))
        ref = tci.HeffPlan(ctx, to_dev(L), to_dev(Wn), to_dev(R), precision=prec)
        out, out_ref = torch.empty_like(dpsi), torch.empty_like(dpsi)
        plan.apply(dpsi, out)
        ref.apply(dpsi, out_ref)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), out_ref.cpu().numpy())
        tol = 1e-12 if prec == "native" else 1e-6
        assert rel_frob_err(out.cpu().numpy(), o_heff.heff_apply(L, Wn, R, psi)) < tol
        for _ in range(3):
            r = plan.lanczos(dpsi, 12, True, x)
            r_ref = ref.lanczos(dpsi, 12, True, torch.empty_like(dpsi))
            assert r["theta"] == r_ref["theta"]
            np.testing.assert_array_equal(r["alpha"], r_ref["alpha"])


def test_plan_reload_error_codes(ctx, tci):
    """tci_heff_plan_reload: a non-F64 tensor is DTYPE, a non-row-major one or another shape is
    SHAPE, and an invalid tensor handle is INVALID_ARG."""
    import ctypes
    import torch
    psi, L, R, W = dense_heff_inputs(16, seed=3)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="native")
    dL, dW, dR = to_dev(L), to_dev(W), to_dev(R)
    with pytest.raises(tci.TciError) as e:
        plan.reload(dL.float(), dW, dR)
    assert e.value.status_name == "TCI_ERR_DTYPE"
    with pytest.raises(tci.TciError) as e:
        plan.reload(dL.transpose(0, 2), dW, dR)
    assert e.value.status_name == "TCI_ERR_SHAPE"
    with pytest.raises(tci.TciError) as e:
        plan.reload(to_dev(dense_heff_inputs(17, seed=3)[1]), dW, dR)
    assert e.value.status_name == "TCI_ERR_SHAPE"
    tw, tr = ctx.wrap(dW), ctx.wrap(dR)
    junk = ctypes.create_string_buffer(4096)             # zero bytes: no tensor handle's magic
    bogus = ctypes.c_void_p(ctypes.addressof(junk))
    st = tci.lib.tci_heff_plan_reload(plan.handle, bogus, tw.handle, None, tr.handle)
    assert tci.STATUS[st] == "TCI_ERR_INVALID_ARG"
    torch.cuda.synchronize()
