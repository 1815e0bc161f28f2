"""Complex (C128) H_eff plans: four native complex contractions vs the oracle."""
import numpy as np
import pytest

from oracle import heff as o_heff
from oracle.contract import rel_frob_err
from tci_synth import complex_heff_inputs, heisenberg_mpo

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("chi,chi_r,Dw,d", [(7, 13, 3, 2), (33, 17, 5, 2), (64, 64, 5, 2), (5, 9, 4, 3)])
def test_complex_heff_matches_oracle(ctx, tci, chi, chi_r, Dw, d):
    import torch
    psi, L, R, W = complex_heff_inputs(chi, 11, chi_r, Dw, d)
    plan = tci.HeffPlan(ctx, _dev(L), _dev(W), _dev(R), precision="native")
    out = torch.full(psi.shape, complex("nan"), dtype=torch.complex128, device="cuda")
    plan.apply(_dev(psi), out)
    torch.cuda.synchronize()
    ref = o_heff.heff_apply(L, W, R, psi)
    assert rel_frob_err(out.cpu().numpy(), ref) < 1e-13
    assert plan.flops == 8.0 * (chi * d * d * chi_r * Dw * (chi + chi_r) + 2.0 * chi * chi_r * d ** 3 * Dw ** 2)


def test_complex_heff_with_a_real_mpo_equals_two_real_matvecs(ctx, tci):
    """H_eff is linear: with real L, W, R the complex matvec acts on Re psi and Im psi separately."""
    import torch
    from tci_synth import dense_heff_inputs
    psi_r, L, R, W = dense_heff_inputs(24, seed=3)
    psi_i = dense_heff_inputs(24, seed=4)[0]
    c = lambda a: _dev(a.astype(np.complex128))
    plan = tci.HeffPlan(ctx, c(L), c(W), c(R), precision="native")
    out = torch.empty(psi_r.shape, dtype=torch.complex128, device="cuda")
    plan.apply(_dev(psi_r + 1j * psi_i), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert rel_frob_err(got.real, o_heff.heff_apply(L, W, R, psi_r)) < 1e-13
    assert rel_frob_err(got.imag, o_heff.heff_apply(L, W, R, psi_i)) < 1e-13


def test_complex_plan_rejects_other_calls(ctx, tci):
    import torch
    psi, L, R, W = complex_heff_inputs(8, 2, 8, 5, 2)
    plan = tci.HeffPlan(ctx, _dev(L), _dev(W), _dev(R), precision="native")
    with pytest.raises(RuntimeError):
        plan.lanczos(_dev(psi.real.copy()), 4)            # F64 start vector on a complex plan
    with pytest.raises(RuntimeError):
        plan.apply(_dev(psi.real.copy()), torch.empty(psi.shape, dtype=torch.float64, device="cuda"))
    with pytest.raises(RuntimeError):
        tci.HeffPlan(ctx, _dev(L), _dev(W.real.copy()), _dev(R), precision="native")


def test_complex_two_site_mpos(ctx, tci):
    import torch
    psi, L, R, W = complex_heff_inputs(9, 5, 12, 4, 2)
    W2 = complex_heff_inputs(2, 6, 2, 4, 2)[3]
    plan = tci.HeffPlan(ctx, _dev(L), _dev(W), _dev(R), precision="native", W2=_dev(W2))
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    plan.apply(_dev(psi), out)
    torch.cuda.synchronize()
    assert rel_frob_err(out.cpu().numpy(), o_heff.heff_apply(L, W, R, psi, W2=W2)) < 1e-13


def _lanczos(tci, ctx, L, W, R, psi, m, gs="dgks"):
    import torch
    plan = tci.HeffPlan(ctx, _dev(L), _dev(W), _dev(R), precision="native")
    plan.set_gram_schmidt(gs)
    x = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    res = plan.lanczos(_dev(psi), m, True, x)
    res["x"] = x.cpu().numpy()
    return res


@pytest.mark.parametrize("gs", ["dgks", "twice"])
def test_complex_lanczos_matches_real_form_oracle(ctx, tci, gs):
    from oracle import lanczos as o_lanczos
    from tci_synth import hermitian_heff_inputs
    psi, L, R, W = hermitian_heff_inputs(8, 3, 6)
    r = _lanczos(tci, ctx, L, W, R, psi, 20, gs)
    o = o_lanczos.lanczos_real_form(lambda v: o_heff.heff_apply(L, W, R, v), psi, 20)
    assert r["steps"] == o["steps"] == 20
    np.testing.assert_allclose(r["alpha"], o["alpha"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(r["beta"], o["beta"], rtol=1e-10, atol=1e-10)
    assert abs(r["theta"] - o["theta"]) < 1e-10 * abs(o["theta"])
    assert np.linalg.norm(r["x"].ravel() - o["x"]) < 1e-8


def test_complex_lanczos_reaches_the_hermitian_ground_energy(ctx, tci):
    from tci_synth import hermitian_heff_inputs
    psi, L, R, W = hermitian_heff_inputs(3, 5, 2)
    H = o_heff.heff_matrix_loops(L, W, R)
    r = _lanczos(tci, ctx, L, W, R, psi, 2 * H.shape[0])
    assert abs(r["theta"] - np.linalg.eigvalsh(H)[0]) < 1e-9
    x = r["x"].ravel()
    assert np.linalg.norm(H @ x - r["theta"] * x) < 1e-7


def test_complex_lanczos_rejects_double_float_vectors(ctx, tci):
    from tci_synth import hermitian_heff_inputs
    psi, L, R, W = hermitian_heff_inputs(4, 3, 4)
    plan = tci.HeffPlan(ctx, _dev(L), _dev(W), _dev(R), precision="native")
    plan.set_lanczos_arith("df32")
    with pytest.raises(RuntimeError):
        plan.lanczos(_dev(psi), 4)
