"""GPU parity of the U(1) block-sparse H_eff (grouped split-BF16) vs the densified FP64 oracle."""
import numpy as np
import pytest

from conftest import to_dev
from oracle import blocksparse as o_bs
from oracle.contract import rel_frob_err
from tci_synth import MPO_CHANNEL_CHARGE, PHYS_CHARGE, blocksparse_inputs, blocksparse_structure

pytestmark = pytest.mark.gpu


def run_bs(tci, ctx, inp, tile_n=None):
    import torch
    dims, qmax = inp["dims"], inp["qmax"]
    st = blocksparse_structure(dims, qmax)
    charges = np.arange(len(dims)) - qmax
    Lp = to_dev(tci.pack_blocks(inp["L"], st["L"]))
    Rp = to_dev(tci.pack_blocks(inp["R"], st["R"]))
    plan = tci.BsHeffPlan(ctx, charges, dims, PHYS_CHARGE, MPO_CHANNEL_CHARGE, Lp, Rp, to_dev(inp["W"]))
    psi = to_dev(tci.pack_blocks(inp["psi"], st["psi"]))
    assert plan.psi_size == psi.numel()
    if tile_n is not None:
        plan.set_tile_n(tile_n)
        assert plan.tile_n == tile_n
    out = torch.full_like(psi, float("nan"))
    plan.apply(psi, out)
    torch.cuda.synchronize()
    shapes = {k: (dims[k[0]], dims[k[3]]) for k in st["psi"]}
    return tci.unpack_blocks(out.cpu().numpy(), st["psi"], shapes), plan, st


def blocks_err(got, ref):
    num = sum(np.sum((got[k].astype(np.float64) - ref[k]) ** 2) for k in ref)
    den = sum(np.sum(ref[k] ** 2) for k in ref)
    return float(np.sqrt(num / den))


@pytest.mark.parametrize("total,qmax,sigma,seed", [(64, 5, 2.0, 3), (300, 9, 3.0, 4), (97, 15, 5.0, 5)])
def test_blocksparse_small_matches_oracle(ctx, tci, total, qmax, sigma, seed):
    inp = blocksparse_inputs(total=total, seed=seed, qmax=qmax, sigma=sigma)
    got, plan, st = run_bs(tci, ctx, inp)
    ref, _ = o_bs.bs_heff_apply(inp)
    assert blocks_err(got, ref) < 1e-6
    assert plan.flops == o_bs.bs_flops(inp)


def test_blocksparse_config_2048(ctx, tci):
    inp = blocksparse_inputs(total=2048, seed=20251223)
    got, plan, st = run_bs(tci, ctx, inp)
    ref, _ = o_bs.bs_heff_apply(inp)
    assert blocks_err(got, ref) < 1e-6
    assert abs(plan.flops - o_bs.bs_flops(inp)) <= 1e-9 * plan.flops


def test_blocksparse_repeat_is_deterministic(ctx, tci):
    inp = blocksparse_inputs(total=200, seed=9, qmax=7, sigma=3.0)
    a, plan, _ = run_bs(tci, ctx, inp)
    b, _, _ = run_bs(tci, ctx, inp)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_blocksparse_graph_replay_with_new_buffers(ctx, tci):
    """Later calls replay a captured CUDA graph; inputs in fresh buffers must be picked up."""
    import torch
    inp = blocksparse_inputs(total=120, seed=12, qmax=6, sigma=2.5)
    dims, qmax = inp["dims"], inp["qmax"]
    st = blocksparse_structure(dims, qmax)
    plan = tci.BsHeffPlan(ctx, np.arange(len(dims)) - qmax, dims, PHYS_CHARGE, MPO_CHANNEL_CHARGE,
                          to_dev(tci.pack_blocks(inp["L"], st["L"])), to_dev(tci.pack_blocks(inp["R"], st["R"])),
                          to_dev(inp["W"]))
    shapes = {k: (dims[k[0]], dims[k[3]]) for k in st["psi"]}
    rng = np.random.default_rng(5)
    keep = []   # every call's buffers stay alive, so each call gets new input and output addresses
    for call in range(4):
        psi_blocks = {k: rng.standard_normal(v.shape).astype(np.float32) for k, v in inp["psi"].items()}
        psi = to_dev(tci.pack_blocks(psi_blocks, st["psi"]))
        out = torch.full_like(psi, float("nan"))
        keep.append((psi, out))
        plan.apply(psi, out)
        torch.cuda.synchronize()
        got = tci.unpack_blocks(out.cpu().numpy(), st["psi"], shapes)
        ref, _ = o_bs.bs_heff_apply(dict(inp, psi=psi_blocks))
        assert blocks_err(got, ref) < 1e-6, call
    assert len({o.data_ptr() for _, o in keep}) == len(keep)


@pytest.mark.parametrize("total,qmax,sigma,seed", [(64, 5, 2.0, 3), (97, 15, 5.0, 5), (2048, 15, 5.0, 20251223)])
def test_blocksparse_narrow_tiles_match_oracle(ctx, tci, total, qmax, sigma, seed):
    """The 128 x 64 tile shape (an autotuner choice) gives the oracle's blocks, including sectors
    wider than one tile and ragged last tiles."""
    inp = blocksparse_inputs(total=total, seed=seed, qmax=qmax, sigma=sigma)
    got, plan, st = run_bs(tci, ctx, inp, tile_n=64)
    ref, _ = o_bs.bs_heff_apply(inp)
    assert blocks_err(got, ref) < 1e-6


def test_blocksparse_autotune_chooses_a_tile_shape(ctx, tci):
    import torch
    inp = blocksparse_inputs(total=300, seed=4, qmax=9, sigma=3.0)
    dims, qmax = inp["dims"], inp["qmax"]
    st = blocksparse_structure(dims, qmax)
    plan = tci.BsHeffPlan(ctx, np.arange(len(dims)) - qmax, dims, PHYS_CHARGE, MPO_CHANNEL_CHARGE,
                          to_dev(tci.pack_blocks(inp["L"], st["L"])), to_dev(tci.pack_blocks(inp["R"], st["R"])),
                          to_dev(inp["W"]))
    psi = to_dev(tci.pack_blocks(inp["psi"], st["psi"]))
    plan.autotune(psi, max_chunk_k=256)
    assert plan.tile_n in (64, 128)
    out = torch.full_like(psi, float("nan"))
    plan.apply(psi, out)
    torch.cuda.synchronize()
    shapes = {k: (dims[k[0]], dims[k[3]]) for k in st["psi"]}
    got = tci.unpack_blocks(out.cpu().numpy(), st["psi"], shapes)
    ref, _ = o_bs.bs_heff_apply(inp)
    assert blocks_err(got, ref) < 1e-6
    with pytest.raises(tci.TciError):
        plan.set_tile_n(96)
    assert plan.ww_variant in (0, 1, 2, 3)
    # a second plan of the same shape takes the cached GEMM configuration (no candidate runs)
    # and still times its W.W variants on its own input
    plan2 = tci.BsHeffPlan(ctx, np.arange(len(dims)) - qmax, dims, PHYS_CHARGE, MPO_CHANNEL_CHARGE,
                           to_dev(tci.pack_blocks(inp["L"], st["L"])), to_dev(tci.pack_blocks(inp["R"], st["R"])),
                           to_dev(inp["W"]))
    assert plan2.autotune(psi, max_chunk_k=256) == plan.autotune(psi, max_chunk_k=256)
    out2 = torch.full_like(psi, float("nan"))
    plan2.apply(psi, out2)
    torch.cuda.synchronize()
    assert blocks_err(tci.unpack_blocks(out2.cpu().numpy(), st["psi"], shapes), ref) < 1e-6


@pytest.mark.parametrize("total,qmax,sigma,seed", [(64, 5, 2.0, 3), (97, 15, 5.0, 5), (2048, 15, 5.0, 20251223)])
def test_blocksparse_ww_variants_agree_bit_for_bit(ctx, tci, total, qmax, sigma, seed):
    """The W.W kernels (shared-memory tiles; 4 x 4 register micro-tiles with vector loads and
    stores over all outputs or groups of them; an autotuner choice) form every element with the same terms in the same order:
    identical outputs, equal to the oracle's blocks.  Sector dims 3..162 leave ragged a' and b
    edges in both tile shapes; the micro-tile writes zeros into the K padding past each sub-block,
    which GEMM2 must see as zeros."""
    import torch
    inp = blocksparse_inputs(total=total, seed=seed, qmax=qmax, sigma=sigma)
    dims, qmax = inp["dims"], inp["qmax"]
    st = blocksparse_structure(dims, qmax)
    plan = tci.BsHeffPlan(ctx, np.arange(len(dims)) - qmax, dims, PHYS_CHARGE, MPO_CHANNEL_CHARGE,
                          to_dev(tci.pack_blocks(inp["L"], st["L"])), to_dev(tci.pack_blocks(inp["R"], st["R"])),
                          to_dev(inp["W"]))
    psi = to_dev(tci.pack_blocks(inp["psi"], st["psi"]))
    outs = []
    for variant in (0, 1, 2, 3, 0):
        plan.set_ww_variant(variant)
        assert plan.ww_variant == variant
        out = torch.full_like(psi, float("nan"))
        plan.apply(psi, out)
        plan.apply(psi, out)          # the second call replays the captured graph
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)
    shapes = {k: (dims[k[0]], dims[k[3]]) for k in st["psi"]}
    ref, _ = o_bs.bs_heff_apply(inp)
    assert blocks_err(tci.unpack_blocks(outs[0], st["psi"], shapes), ref) < 1e-6
    with pytest.raises(tci.TciError):
        plan.set_ww_variant(4)
