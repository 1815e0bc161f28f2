"""GPU parity of the batched TEBD theta (split-BF16 grouped GEMM with the gate in its epilogue) vs the
complex128 oracle."""
import numpy as np
import pytest

from conftest import to_dev
from oracle import tebd as o_tebd
from oracle.contract import rel_frob_err
from tci_synth import tebd_inputs

pytestmark = pytest.mark.gpu


def run_tebd(tci, ctx, chis, A, B, G, precision="split_bf16", tile_n=None):
    import torch
    plan = tci.TebdPlan(ctx, chis, precision=precision)
    if tile_n is not None:
        plan.set_tile_n(tile_n)
        assert plan.tile_n == tile_n
    pa = to_dev(np.concatenate([a.ravel() for a in A]))
    pb = to_dev(np.concatenate([b.ravel() for b in B]))
    pg = to_dev(np.concatenate([g.ravel() for g in G]))
    th = torch.full((sum(4 * c * c for c in chis),), complex("nan+nanj"), dtype=torch.complex64, device="cuda")
    plan.apply(pa, pb, pg, th)
    torch.cuda.synchronize()
    th = th.cpu().numpy()
    out, off = [], 0
    for c in chis:
        out.append(th[off:off + 4 * c * c].reshape(c, 2, 2, c))
        off += 4 * c * c
    return out, plan


@pytest.mark.parametrize("nb,lo,hi,seed", [(5, 3, 9, 1), (17, 16, 130, 2), (3, 1, 1, 3)])
def test_tebd_small_matches_oracle(ctx, tci, nb, lo, hi, seed):
    chis, A, B, G = tebd_inputs(nb, seed=seed, chi_lo=lo, chi_hi=hi)
    got, plan = run_tebd(tci, ctx, chis, A, B, G)
    for g_, a, b, gg in zip(got, A, B, G):
        assert rel_frob_err(g_, o_tebd.theta(a, b, gg)) < 1e-5
    assert plan.flops == o_tebd.tebd_flops(chis)


def test_tebd_config_256_bonds(ctx, tci):
    chis, A, B, G = tebd_inputs(256, seed=20251223)
    got, plan = run_tebd(tci, ctx, chis, A, B, G)
    num = den = 0.0
    worst = 0.0
    for g_, a, b, gg in zip(got, A, B, G):
        ref = o_tebd.theta(a, b, gg)
        e = np.sum(np.abs(g_ - ref) ** 2)
        num += e
        den += np.sum(np.abs(ref) ** 2)
        worst = max(worst, np.sqrt(e / np.sum(np.abs(ref) ** 2)))
    assert np.sqrt(num / den) < 1e-5 and worst < 1e-5
    assert abs(plan.flops - o_tebd.tebd_flops(chis)) <= 1e-9 * plan.flops


def test_tebd_unitary_gate_preserves_norm(ctx, tci):
    chis, A, B, G = tebd_inputs(8, seed=4, chi_lo=20, chi_hi=60)
    got, _ = run_tebd(tci, ctx, chis, A, B, G)
    eye = [np.eye(4, dtype=np.complex64).reshape(2, 2, 2, 2)] * len(chis)
    plain, _ = run_tebd(tci, ctx, chis, A, B, eye)
    for g_, p_ in zip(got, plain):
        assert abs(np.linalg.norm(g_) - np.linalg.norm(p_)) < 1e-5 * np.linalg.norm(p_)


def test_tebd_graph_replay_with_new_buffers(ctx, tci):
    """Later calls replay a captured CUDA graph with updated pointer arguments."""
    import torch
    chis = [9, 33, 70, 5]
    plan = tci.TebdPlan(ctx, chis)
    for call, seed in enumerate((21, 22, 23)):
        _, A, B, G = tebd_inputs(len(chis), seed=seed, chi_lo=1, chi_hi=1)
        rng = np.random.default_rng(seed)
        A = [(rng.standard_normal((c, 2, c)) + 1j * rng.standard_normal((c, 2, c))).astype(np.complex64) for c in chis]
        B = [(rng.standard_normal((c, 2, c)) + 1j * rng.standard_normal((c, 2, c))).astype(np.complex64) for c in chis]
        G = G[:1] * len(chis)
        pa = to_dev(np.concatenate([a.ravel() for a in A]))
        pb = to_dev(np.concatenate([b.ravel() for b in B]))
        pg = to_dev(np.concatenate([g.ravel() for g in G]))
        th = torch.full((sum(4 * c * c for c in chis),), complex("nan+nanj"), dtype=torch.complex64, device="cuda")
        plan.apply(pa, pb, pg, th)
        torch.cuda.synchronize()
        th = th.cpu().numpy()
        off = 0
        for c, a, b, g in zip(chis, A, B, G):
            assert rel_frob_err(th[off:off + 4 * c * c].reshape(c, 2, 2, c), o_tebd.theta(a, b, g)) < 1e-5, call
            off += 4 * c * c


def test_tebd_theta_batched_on_handles(ctx, tci):
    """The handle form (tci_tebd_theta_batched) equals the oracle bond by bond."""
    chis, A, B, G = tebd_inputs(7, seed=8, chi_lo=3, chi_hi=70)
    ctx.set_precision("split_bf16")
    try:
        out = tci.tebd_theta_batched(ctx, [to_dev(a) for a in A], [to_dev(b) for b in B], [to_dev(g) for g in G])
    finally:
        ctx.set_precision("native")
    for t, a, b, g in zip(out, A, B, G):
        got = t.to_numpy()
        assert got.shape == (a.shape[0], 2, 2, a.shape[0])
        assert rel_frob_err(got, o_tebd.theta(a, b, g)) < 1e-5


@pytest.mark.parametrize("nb,lo,hi,seed", [(5, 3, 9, 1), (17, 16, 130, 2), (40, 16, 512, 20251223)])
def test_tebd_narrow_tiles_match_oracle(ctx, tci, nb, lo, hi, seed):
    """The 128 x 64 tile shape (an autotuner choice) gives the oracle's theta for every bond."""
    chis, A, B, G = tebd_inputs(nb, seed=seed, chi_lo=lo, chi_hi=hi)
    got, plan = run_tebd(tci, ctx, chis, A, B, G, tile_n=64)
    for g_, a, b, gg in zip(got, A, B, G):
        assert rel_frob_err(g_, o_tebd.theta(a, b, gg)) < 1e-5


def test_tebd_three_products_match_oracle(ctx, tci):
    """SPLIT_BF16_3 (hi*hi, hi*mid, mid*hi per real product) through the gate epilogue: both
    accumulation paths (chi <= 256 fits one hi*hi chunk, chi > 256 does not)."""
    chis, A, B, G = tebd_inputs(12, seed=31, chi_lo=40, chi_hi=400)
    got, _ = run_tebd(tci, ctx, chis, A, B, G, precision="split_bf16_3")
    for g_, a, b, gg in zip(got, A, B, G):
        assert rel_frob_err(g_, o_tebd.theta(a, b, gg)) < 1e-4


def test_tebd_misaligned_gate_is_rejected(ctx, tci):
    """The gate epilogue reads G as 16-byte vectors: a G base that is only 8-byte aligned is
    refused on the host (TCI_ERR_INVALID_ARG) before anything launches."""
    import torch
    chis, A, B, G = tebd_inputs(2, seed=5, chi_lo=4, chi_hi=6)
    plan = tci.TebdPlan(ctx, chis)
    pa = to_dev(np.concatenate([a.ravel() for a in A]))
    pb = to_dev(np.concatenate([b.ravel() for b in B]))
    pg = to_dev(np.concatenate([np.zeros(1, np.complex64)] + [g.ravel() for g in G]))[1:]
    th = torch.zeros(sum(4 * c * c for c in chis), dtype=torch.complex64, device="cuda")
    assert pg.data_ptr() % 16 == 8
    with pytest.raises(tci.TciError) as ei:
        plan.apply(pa, pb, pg, th)
    assert ei.value.status_name == "TCI_ERR_INVALID_ARG"


def test_tebd_config_256_bonds_chunk512(ctx, tci):
    """The 256-bond batch with a 512-deep hi*hi accumulation chunk (the TEBD row's tuner may pick
    it: theta's bound is 1e-5) stays within 1e-5 of the oracle, aggregate and worst bond."""
    chis, A, B, G = tebd_inputs(256, seed=20251223)
    ctx.set_split_chunks(512, 4096)
    try:
        got, _ = run_tebd(tci, ctx, chis, A, B, G)
    finally:
        ctx.set_split_chunks(256, 1024)
    num = den = worst = 0.0
    for g_, a, b, gg in zip(got, A, B, G):
        ref = o_tebd.theta(a, b, gg)
        e = np.sum(np.abs(g_ - ref) ** 2)
        num += e
        den += np.sum(np.abs(ref) ** 2)
        worst = max(worst, np.sqrt(e / np.sum(np.abs(ref) ** 2)))
    assert np.sqrt(num / den) < 1e-5 and worst < 1e-5
