"""Autotuner (plan configuration search + cache) keeps parity and reuses cached choices."""
import os

import numpy as np
import pytest

from conftest import to_dev
from oracle import heff as o_heff, tebd as o_tebd
from oracle.contract import rel_frob_err
from tci_synth import dense_heff_inputs, tebd_inputs

pytestmark = pytest.mark.gpu


def test_heff_autotune_parity_and_cache(ctx, tci, tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("TCI_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    psi, L, R, W = dense_heff_inputs(256, seed=31)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="split_bf16")
    dpsi = to_dev(psi)
    out = torch.empty_like(dpsi)
    chunk, xchunk, raster = plan.autotune(dpsi, out, max_chunk_k=256)
    assert chunk in (128, 256) and xchunk in (1024, 4096) and raster in (0, 8, 16)
    plan.apply(dpsi, out)
    torch.cuda.synchronize()
    assert rel_frob_err(out.cpu().numpy(), o_heff.heff_apply(L, W, R, psi)) < 1e-6
    # same shape again: answered from the cache
    plan2 = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="split_bf16")
    assert plan2.autotune(dpsi, out, max_chunk_k=256) == (chunk, xchunk, raster)


def test_tebd_autotune_parity(ctx, tci):
    import torch
    chis, A, B, G = tebd_inputs(6, seed=32, chi_lo=20, chi_hi=150)
    plan = tci.TebdPlan(ctx, chis)
    pa = to_dev(np.concatenate([a.ravel() for a in A]))
    pb = to_dev(np.concatenate([b.ravel() for b in B]))
    pg = to_dev(np.concatenate([g.ravel() for g in G]))
    th = torch.empty(sum(4 * c * c for c in chis), dtype=torch.complex64, device="cuda")
    cfg = plan.autotune(pa, pb, pg, th, max_chunk_k=256)
    assert cfg[0] in (128, 256)
    th.fill_(complex("nan+nanj"))
    plan.apply(pa, pb, pg, th)
    torch.cuda.synchronize()
    got = th.cpu().numpy()
    off = 0
    for c, a, b, g in zip(chis, A, B, G):
        assert rel_frob_err(got[off:off + 4 * c * c].reshape(c, 2, 2, c), o_tebd.theta(a, b, g)) < 1e-5
        off += 4 * c * c


def test_heff_every_tuning_candidate_chi2048(ctx, tci):
    """At chi = 2048 every configuration the tuner may pick keeps the 1e-6 matvec bound."""
    import torch
    psi, L, R, W = dense_heff_inputs(2048, seed=20251223)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="split_bf16")
    ref = o_heff.heff_apply(L, W, R, psi)
    dpsi = to_dev(psi)
    out = torch.empty_like(dpsi)
    for chunk in (128, 256):
        for xchunk in (1024, 4096):
            for raster in (0, 8, 16):
                for ww_na in (2, 4):
                    plan.set_config(chunk, xchunk, raster, ww_na)
                    out.fill_(float("nan"))
                    plan.apply(dpsi, out)
                    torch.cuda.synchronize()
                    err = rel_frob_err(out.cpu().numpy(), ref)
                    assert err < 1e-6, (chunk, xchunk, raster, ww_na, err)
