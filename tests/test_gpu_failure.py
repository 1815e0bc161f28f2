"""Failure detection without a GPU fault: an expired bounded wait is reported and the context recovers.

The tensor-core kernel bounds every wait on work in flight; a context wait
limit of 1 ns makes its first wait on a TMA copy expire.  The kernel then
lets its copies and MMAs land, frees tensor memory and returns, and the next
synchronising call reports TCI_ERR_TIMEOUT.  Nothing faults or hangs.
"""
import numpy as np
import pytest

from conftest import to_dev
from oracle import heff as o_heff
from oracle.contract import contract as o_contract, rel_frob_err
from tci_synth import dense_heff_inputs, random_tensor

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_context_recovers(ctx, tci):
    A = random_tensor([300, 200], 1)
    B = random_tensor([200, 260], 2)
    ctx.set_precision("split_bf16")
    try:
        ctx.set_wait_limit(1)
        with pytest.raises(tci.TciError) as ei:
            tci.contract(ctx, to_dev(A), "ij", to_dev(B), "jk", "ik")
            ctx.synchronize()
        assert ei.value.status_name == "TCI_ERR_TIMEOUT"
        ctx.set_wait_limit(0)
        ctx.synchronize()                                # the status was reported once; nothing pending
        out = tci.contract(ctx, to_dev(A), "ij", to_dev(B), "jk", "ik")
        ctx.synchronize()
        assert rel_frob_err(out.cpu().numpy(), o_contract(A, "ij", B, "jk", "ik")) < 1e-6
    finally:
        ctx.set_wait_limit(0)
        ctx.set_precision("native")


def test_expired_wait_in_heff_plan_then_recovery(ctx, tci):
    import torch
    psi, L, R, W = dense_heff_inputs(96, seed=12)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="split_bf16")
    dpsi = to_dev(psi)
    out = torch.empty_like(dpsi)
    try:
        ctx.set_wait_limit(1)
        with pytest.raises(tci.TciError) as ei:
            plan.apply(dpsi, out)
            ctx.synchronize()
        assert ei.value.status_name == "TCI_ERR_TIMEOUT"
    finally:
        ctx.set_wait_limit(0)
    plan.apply(dpsi, out)
    ctx.synchronize()
    assert rel_frob_err(out.cpu().numpy(), o_heff.heff_apply(L, W, R, psi)) < 1e-6
    ctx.set_precision("native")
