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


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("gs", ["dgks", "twice"])
def test_lanczos_basis_beyond_one_pass_matches_oracle(ctx, tci, arith, gs):
    """chi = 128 (n = 2^16), 32 steps: from step 7 on the vector work runs as separate passes, and
    from step 20 on the basis (over 20 vectors) is updated and projected in groups of passes, each
    forming its dot and norm totals in its last block; alpha, beta, theta and the Ritz vector
    equal the oracle's."""
    psi, L, R, W = dense_heff_inputs(128, seed=31)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 32, arith=arith, gs=gs)
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 32)
    assert r["steps"] == o["steps"] == 32
    np.testing.assert_allclose(r["alpha"], o["alpha"], rtol=1e-9, atol=1e-9 * np.abs(o["alpha"]).max())
    np.testing.assert_allclose(r["beta"], o["beta"], rtol=1e-9, atol=1e-9 * np.abs(o["beta"]).max())
    assert abs(r["theta"] - o["theta"]) < 1e-10 * abs(o["theta"])
    assert np.linalg.norm(r["x"].ravel() - o["x"]) < 1e-7


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


def test_lanczos_chi2048_timed_configuration(ctx, tci):
    """The timed solve itself: autotuned split-BF16 plan, 20 DGKS steps at chi = 2048.

    The oracle's own 20-step solve is too slow here, so the result is checked through
    properties that hold at any size, each against FP64 arithmetic outside the GPU path:
      - x is a unit vector;
      - theta is the lowest eigenvalue of the returned tridiagonal T (Sturm bisection) and
        lies below every alpha_j (each alpha_j is a Rayleigh quotient in the Krylov space);
      - theta equals the FP64 Rayleigh quotient <x, H x>, H x taken by one oracle matvec;
      - ||H x - theta x|| equals the Lanczos residual beta_m |y_m| (H V = V T + beta_m v e_m^T).
    The split-BF16 matvec error bound (1e-6 relative) sets both tolerances.
    """
    import torch
    psi, L, R, W = dense_heff_inputs(2048, seed=20251223)
    dpsi = to_dev(psi)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="split_bf16")
    out = torch.empty_like(dpsi)
    plan.autotune(dpsi, out, max_chunk_k=256)
    x = torch.empty_like(dpsi)
    r = plan.lanczos(dpsi, 20, True, x)
    x = x.cpu().numpy().ravel()
    a, b, theta = r["alpha"], r["beta"], r["theta"]
    assert r["steps"] == 20
    assert abs(np.linalg.norm(x) - 1.0) < 1e-12
    assert abs(theta - o_lanczos.lowest_eigenvalue_bisect(a, b[:-1])) < 1e-12 * abs(theta)
    assert theta <= a.min()
    hx = o_heff.heff_apply(L, W, R, x.reshape(psi.shape)).ravel()
    rq = float(x @ hx)
    assert abs(rq - theta) < 1e-6 * abs(theta), (rq, theta)
    y = o_lanczos.tridiag_eigvec(a, b[:-1], theta)
    res_true = np.linalg.norm(hx - theta * x)
    res_lanczos = abs(b[-1] * y[-1]) / np.linalg.norm(y)
    assert abs(res_true - res_lanczos) < 1e-6 * abs(theta), (res_true, res_lanczos)
    st = plan.lanczos_stats()
    assert st["steps"] == 20 and 1 <= st["fused_pass3"] <= st["second_passes"], st
    assert st["df_term_passes"] >= 1, st   # matvec-error-level terms from j = 7 on


def test_lanczos_rounding_level_terms_counted(ctx, tci):
    """FP64 plan, FP64 vectors, vectors of 2^20 elements (chi = 512): from step 2 on the
    rounding-level update terms take the FP32 path and every repeated projection is folded
    into the next-vector pass, with alpha, beta and theta still equal to the oracle's; shorter
    vectors and double-float vectors take neither."""
    import torch
    psi, L, R, W = dense_heff_inputs(512, seed=20251223)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="native")
    plan.set_gram_schmidt("twice")
    x = torch.empty(psi.shape, dtype=torch.float64, device="cuda")
    r = plan.lanczos(to_dev(psi), 20, True, x)
    st = plan.lanczos_stats()
    assert st == {"steps": 20, "second_passes": 20, "f32_term_passes": 18, "df_term_passes": 0, "fused_pass3": 20}, st
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    np.testing.assert_allclose(r["alpha"], o["alpha"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(r["beta"], o["beta"], rtol=1e-10, atol=1e-10)
    assert abs(r["theta"] - o["theta"]) < 1e-12 * abs(o["theta"])
    plan.set_lanczos_arith("df32")
    plan.lanczos(to_dev(psi), 20, True, x)
    st = plan.lanczos_stats()
    assert st["steps"] == 20 and st["f32_term_passes"] + st["df_term_passes"] + st["fused_pass3"] == 0, st
    small, Ls, Rs, Ws = dense_heff_inputs(32, seed=20251223)
    plan_s = tci.HeffPlan(ctx, to_dev(Ls), to_dev(Ws), to_dev(Rs), precision="native")
    xs = torch.empty(small.shape, dtype=torch.float64, device="cuda")
    plan_s.lanczos(to_dev(small), 20, True, xs)
    st = plan_s.lanczos_stats()
    assert st["f32_term_passes"] + st["df_term_passes"] == 0, st


@pytest.mark.parametrize("precision,chi,chi_r,arith", [
    ("split_bf16", 64, 64, "f64"), ("split_bf16", 75, 61, "f64"), ("split_bf16", 64, 40, "df32"),
    ("native", 64, 64, "f64"), ("native", 75, 61, "f64"), ("native", 64, 40, "df32")])
def test_lanczos_graph_replay_identical(ctx, tci, precision, chi, chi_r, arith):
    """Eager, captured and replayed solves give bit-identical results on split-BF16 and FP64
    plans, with FP64 and double-float vectors, while the start-vector and Ritz-vector buffers
    alternate (the replay patches psi0 and x into the captured kernel nodes); every solve after
    the first eager one runs as a graph launch."""
    import torch
    psi, L, R, W = dense_heff_inputs(chi, seed=13, chi_r=chi_r)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision=precision)
    plan.set_lanczos_arith(arith)
    d1, d2 = to_dev(psi), to_dev(psi)
    x1, x2 = torch.empty_like(d1), torch.empty_like(d1)

    def solve(dpsi, x):
        x.fill_(float("nan"))
        r = plan.lanczos(dpsi, 20, True, x)
        return r, x.cpu().numpy()

    plan.set_lanczos_graphs(False)
    ref, xref = solve(d1, x1)
    assert not plan.lanczos_graph_info()["last_from_graph"]
    plan.set_lanczos_graphs(True)
    for i, (dpsi, x) in enumerate(((d1, x1), (d1, x1), (d1, x2), (d1, x1), (d2, x2), (d2, x1), (d2, x2),
                                   (d1, x2), (d1, x1))):
        r, xr = solve(dpsi, x)
        info = plan.lanczos_graph_info()
        assert info["enabled"] and info["last_from_graph"] == (i >= 1), (i, info)
        assert r["theta"] == ref["theta"] and r["steps"] == ref["steps"]
        np.testing.assert_array_equal(r["alpha"], ref["alpha"])
        np.testing.assert_array_equal(r["beta"], ref["beta"])
        np.testing.assert_array_equal(xr, xref)
    assert plan.lanczos_graph_info()["graph_launches"] == 8


@pytest.mark.parametrize("gs", ["dgks", "twice"])
def test_lanczos_short_and_long_step_paths_mix(ctx, tci, gs):
    """chi = 128 (n = 2^16): the first steps run as one cluster launch each (n (j + 2) <= 2^19),
    the later ones as the multi-kernel passes; alpha, beta, theta equal the oracle's."""
    psi, L, R, W = dense_heff_inputs(128, seed=9)
    r = gpu_lanczos(tci, ctx, L, W, R, psi, 20, gs=gs)
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    assert r["steps"] == o["steps"] == 20
    np.testing.assert_allclose(r["alpha"], o["alpha"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(r["beta"], o["beta"], rtol=1e-10, atol=1e-10)
    assert abs(r["theta"] - o["theta"]) < 1e-12 * abs(o["theta"])
    assert abs(np.linalg.norm(r["x"]) - 1.0) < 1e-12


@pytest.mark.parametrize("precision,chi", [("split_bf16", 512), ("native", 512)])
def test_lanczos_reduced_terms_equal_fp64_terms(ctx, tci, precision, chi):
    """Vectors of 2^20 elements: the FP32 / double-float small update terms change alpha, beta
    and theta only at rounding level against every update term in FP64 (the same plan)."""
    import torch
    psi, L, R, W = dense_heff_inputs(chi, seed=17)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision=precision)
    plan.set_gram_schmidt("twice")
    dpsi = to_dev(psi)
    x = torch.empty_like(dpsi)
    r1 = plan.lanczos(dpsi, 20, True, x)
    st = plan.lanczos_stats()
    assert st["f32_term_passes"] + st["df_term_passes"] >= 12 and st["fused_pass3"] == 20, st
    x1 = x.cpu().numpy()
    plan.set_lanczos_reduced_terms(False)
    r0 = plan.lanczos(dpsi, 20, True, x)
    st = plan.lanczos_stats()
    assert st["f32_term_passes"] + st["df_term_passes"] + st["fused_pass3"] == 0, st
    np.testing.assert_allclose(r1["alpha"], r0["alpha"], rtol=1e-11, atol=1e-11 * np.abs(r0["alpha"]).max())
    np.testing.assert_allclose(r1["beta"], r0["beta"], rtol=1e-11)
    assert abs(r1["theta"] - r0["theta"]) < 1e-12 * abs(r0["theta"])
    assert np.linalg.norm(x1 - x.cpu().numpy()) < 1e-9


@pytest.mark.parametrize("chi,chi_r", [(64, 64), (75, 61), (200, 131)])
def test_lanczos_fused_dots_equal_separate_pass(ctx, tci, chi, chi_r):
    """Split-BF16 plan, FP64 vectors: the first projection's dots formed in the matvec's GEMM2
    epilogue (opt-in) give alpha, beta, theta and the Ritz vector of the separate dot pass up to
    FP64 summation order; ragged shapes exercise partial tiles and partial column groups."""
    import torch
    psi, L, R, W = dense_heff_inputs(chi, seed=21, chi_r=chi_r)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="split_bf16")
    plan.set_lanczos_fused_dots(True)
    plan.set_lanczos_shadow_dots(False)                # both sides form every first-projection dot in FP64
    dpsi = to_dev(psi)
    x = torch.empty_like(dpsi)
    r1 = plan.lanczos(dpsi, 20, True, x)
    x1 = x.cpu().numpy()
    r1b = plan.lanczos(dpsi, 20, True, x)          # captured into a graph and launched
    assert r1b["theta"] == r1["theta"]
    plan.set_lanczos_fused_dots(False)
    r0 = plan.lanczos(dpsi, 20, True, x)
    assert r0["steps"] == r1["steps"] == 20
    np.testing.assert_allclose(r1["alpha"], r0["alpha"], rtol=1e-12, atol=1e-12 * np.abs(r0["alpha"]).max())
    np.testing.assert_allclose(r1["beta"], r0["beta"], rtol=1e-11)
    assert abs(r1["theta"] - r0["theta"]) < 1e-12 * abs(r0["theta"])
    assert np.linalg.norm(x1 - x.cpu().numpy()) < 1e-9
    # and the solve is the FP64 oracle's to the split matvec's error level
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    assert abs(r1["theta"] - o["theta"]) < 1e-6 * abs(o["theta"])


@pytest.mark.parametrize("chi,chi_r", [(64, 64), (75, 61), (256, 256)])
def test_lanczos_shadow_dots_equal_fp64_pass(ctx, tci, chi, chi_r):
    """Split-BF16 plan, FP64 vectors: the double-float Gram-Schmidt dots (opt-in) against the FP64
    dot passes (the default).  The first step (same v_0, same matvec) agrees to
    ~1e-14; later steps agree only to the split matvec's own error level, because the matvec rounds
    its input to FP32 and a 1e-14 change in v can flip such a rounding; theta stays the oracle's to
    that level either way.  Odd column counts take the element-wise next-vector paths; repeated
    solves replay the captured graph bit for bit."""
    import torch
    psi, L, R, W = dense_heff_inputs(chi, seed=23, chi_r=chi_r)
    plan = tci.HeffPlan(ctx, to_dev(L), to_dev(W), to_dev(R), precision="split_bf16")
    dpsi = to_dev(psi)
    x = torch.empty_like(dpsi)
    plan.set_lanczos_shadow_dots(True)
    r1 = plan.lanczos(dpsi, 20, True, x)
    x1 = x.cpu().numpy()
    for _ in range(2):
        r1b = plan.lanczos(dpsi, 20, True, x)
        assert r1b["theta"] == r1["theta"]
        np.testing.assert_array_equal(x.cpu().numpy(), x1)
    plan.set_lanczos_shadow_dots(False)
    r0 = plan.lanczos(dpsi, 20, True, x)
    assert r0["steps"] == r1["steps"] == 20
    assert abs(r1["alpha"][0] - r0["alpha"][0]) < 1e-13 * np.abs(r0["alpha"]).max()
    assert abs(r1["beta"][0] - r0["beta"][0]) < 1e-13 * r0["beta"][0]
    np.testing.assert_allclose(r1["alpha"], r0["alpha"], rtol=1e-5, atol=1e-5 * np.abs(r0["alpha"]).max())
    mv = lambda v: o_heff.heff_apply(L, W, R, v.reshape(psi.shape))
    o = o_lanczos.lanczos(mv, psi, 20)
    for r in (r0, r1):
        assert abs(r["theta"] - o["theta"]) < 1e-6 * abs(o["theta"])
