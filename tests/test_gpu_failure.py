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


def test_injected_allocation_failure_trim_retry_then_alloc_error(tci, monkeypatch, capfd):
    """TCI_FAULT_ALLOC injects out-of-memory answers on the host (the device is never touched):
    one injected failure is absorbed by the pool's trim-and-retry path and the call succeeds;
    two in a row make the call return TCI_ERR_ALLOC, and the context keeps working after it."""
    import torch
    x = to_dev(random_tensor([64, 33], 5))
    ref = x.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    monkeypatch.setenv("TCI_VERBOSE", "1")
    monkeypatch.setenv("TCI_FAULT_ALLOC", "0:1")
    c1 = tci.Context(0, stream)
    y = c1.wrap(x).copy()                               # the context's first pooled allocation
    c1.synchronize()
    np.testing.assert_array_equal(y.to_numpy(), ref)
    assert "pool trimmed, retrying once" in capfd.readouterr().err
    y.free()
    c1.close()
    monkeypatch.setenv("TCI_FAULT_ALLOC", "0:2")
    c2 = tci.Context(0, stream)
    with pytest.raises(tci.TciError) as ei:
        c2.wrap(x).copy()
    assert ei.value.status_name == "TCI_ERR_ALLOC"
    err = capfd.readouterr().err
    assert "pool trimmed, retrying once" in err and "[tci] error 6:" in err
    y = c2.wrap(x).copy()                               # allocation 1 is not injected
    c2.synchronize()
    np.testing.assert_array_equal(y.to_numpy(), ref)
    y.free()
    c2.close()


@pytest.mark.parametrize("level", [0, 1, 2])
def test_verbose_levels(tci, monkeypatch, capfd, level):
    """TCI_VERBOSE (App. C.3): 0 prints nothing, 1 one line per call on stderr, 2 adds the
    call's device time."""
    import re
    import torch
    monkeypatch.setenv("TCI_VERBOSE", str(level))
    monkeypatch.delenv("TCI_FAULT_ALLOC", raising=False)
    a, b = to_dev(random_tensor([12, 2, 9], 1)), to_dev(random_tensor([9, 2, 5], 2))
    capfd.readouterr()
    c = tci.Context(0, torch.cuda.current_stream().cuda_stream)
    tci.contract(c, a, "ijk", b, "klm", "ijlm")
    c.synchronize()
    c.close()
    lines = [ln for ln in capfd.readouterr().err.splitlines() if ln.startswith("[tci]")]
    if level == 0:
        assert lines == []
        return
    assert lines[0].startswith("[tci] create_context device=0")
    assert lines[-1] == "[tci] destroy_context"
    calls = [ln for ln in lines if ln.startswith("[tci] contract ")]
    assert len(calls) == 1 and "ijk,klm->ijlm f64{12,2,9} x f64{9,2,5}" in calls[0]
    if level == 2:
        assert re.search(r" time=\d+\.\d{3} ms$", calls[0]), calls[0]
    else:
        assert "time=" not in calls[0]
