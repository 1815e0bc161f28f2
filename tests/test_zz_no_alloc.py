"""The allocation-free H_eff entry point against the regular plan-based one.

tci_heff_apply_noalloc serves callers that may not allocate device memory
when they apply H_eff; it keeps its intermediates in a fixed array inside
the library.  This file is collected last so that a stop-at-first-failure run
has executed every other test before it.
"""
import ctypes

import numpy as np
import pytest

from conftest import to_dev
from oracle.contract import rel_frob_err
from tci_synth import dense_heff_inputs

pytestmark = pytest.mark.gpu


def _noalloc(tci, L, W, R, psi, out, stream):
    return tci.lib.tci_heff_apply_noalloc(ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                          ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(psi.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), L.shape[0], R.shape[0],
                                          ctypes.c_void_p(stream))


def test_noalloc_matches_plan_path_twice(tci):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    ctx = tci.Context(0, stream)
    # two calls in a row with different sizes and data: the second must not
    # see anything left in the shared scratch by the first
    for chi, chi_r, seed in ((64, 48, 3), (37, 91, 4)):
        psi, L, R, W = dense_heff_inputs(chi, seed=seed, chi_r=chi_r)
        dL, dW, dR, dpsi = to_dev(L), to_dev(W), to_dev(R), to_dev(psi)
        ref = torch.empty_like(dpsi)
        plan = tci.HeffPlan(ctx, dL, dW, dR, precision="native")
        plan.apply(dpsi, ref)
        out = torch.full_like(dpsi, float("nan"))
        assert _noalloc(tci, dL, dW, dR, dpsi, out, stream) == 0, tci.lib.tci_last_error(None)
        torch.cuda.synchronize()
        assert rel_frob_err(out.cpu().numpy(), ref.cpu().numpy()) < 1e-12
        plan.close()
    ctx.close()


def test_noalloc_rejects_oversize(tci):
    import torch
    big = 200   # 200 * 200 > 13094
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = tci.lib.tci_heff_apply_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                        ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                        ctypes.c_void_p(t.data_ptr()), big, big, None)
    assert tci.STATUS[st] == "TCI_ERR_UNSUPPORTED"
    assert b"13094" in tci.lib.tci_last_error(None)
