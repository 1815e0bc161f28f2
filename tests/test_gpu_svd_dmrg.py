"""Device TCI svd / trunc_svd (one-sided Jacobi) and the two-site DMRG sweep against the oracle and ED."""
import numpy as np
import pytest

from conftest import to_dev
from oracle import dmrg as o_dmrg
from oracle import linalg as o_linalg
from tci_synth import heisenberg_mpo, random_tensor

pytestmark = pytest.mark.gpu


def _tensor(tci, ctx, a):
    code = {np.float64: 1, np.float32: 0}[a.dtype.type]
    t = tci.allocate(ctx, a.shape, code)
    t.from_numpy(a)
    return t


def _check_svd(a, k, u, s, vt, tol):
    I = int(np.prod(a.shape[:k]))
    m = a.reshape(I, -1).astype(np.float64)
    kappa = s.shape[0]
    um, vm = u.reshape(I, kappa).astype(np.float64), vt.reshape(kappa, -1).astype(np.float64)
    scale = max(1.0, np.linalg.norm(m))
    assert np.linalg.norm(um * s @ vm - m) < tol * scale                 # reconstruction
    nz = s > tol * s.max() if s.size else s > 0
    np.testing.assert_allclose(um[:, nz].T @ um[:, nz], np.eye(nz.sum()), atol=tol * 10)
    np.testing.assert_allclose(vm[nz] @ vm[nz].T, np.eye(nz.sum()), atol=tol * 10)
    assert np.all(np.diff(s) <= 1e-12 * max(1.0, s.max(initial=0)))


@pytest.mark.parametrize("shape,k", [((3, 4, 12), 2), ((40, 7), 1), ((7, 40), 1), ((33, 2, 2, 17), 2),
                                     ((1, 5), 1), ((64, 2, 2, 64), 2), ((5, 1), 1),
                                     # around the single-launch limits: Jacobi sweeps for vectors <= 64
                                     # long, the pivoted QR for columns <= 256 long
                                     ((64, 64), 1), ((65, 65), 1), ((257, 40), 1), ((40, 257), 1),
                                     ((256, 33), 1)])
def test_svd_matches_oracle(ctx, tci, shape, k):
    a = random_tensor(shape, 21)
    u, s, vt = tci.svd(ctx, _tensor(tci, ctx, a), k)
    u, s, vt = u.to_numpy(), s.to_numpy(), vt.to_numpy()
    ru, rs, rvt = o_linalg.svd(a, k)
    assert u.shape == ru.shape and s.shape == rs.shape and vt.shape == rvt.shape
    np.testing.assert_allclose(s, rs, rtol=1e-12, atol=1e-13)
    _check_svd(a, k, u, s, vt, 1e-12)


def test_svd_rank_deficient_and_f32(ctx, tci):
    rng = np.random.default_rng(5)
    a = rng.standard_normal((30, 3)) @ rng.standard_normal((3, 20))          # rank 3
    u, s, vt = tci.svd(ctx, _tensor(tci, ctx, a), 1)
    s = s.to_numpy()
    np.testing.assert_allclose(s[:3], np.linalg.svd(a, compute_uv=False)[:3], rtol=1e-12)
    assert np.all(s[3:] < 1e-12 * s[0])
    _check_svd(a, 1, u.to_numpy(), s, vt.to_numpy(), 1e-12)
    b = random_tensor((24, 18), 6, np.float32)
    u, s, vt = tci.svd(ctx, _tensor(tci, ctx, b), 1)
    np.testing.assert_allclose(s.to_numpy(), np.linalg.svd(b.astype(np.float64), compute_uv=False), rtol=1e-6)


def test_trunc_svd_rules_match_oracle(ctx, tci):
    s0 = np.array([4.0, 2.0, 1.0, 0.5, 1e-3, 1e-9])
    rng = np.random.default_rng(3)
    q1, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    q2, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    m = np.zeros((6, 8))
    m[:6, :6] = np.diag(s0)
    a = q1 @ m @ q2.T
    tot = float(np.sum(s0 ** 2))
    cases = [(1, 3, 0.0, 0.0), (1, 10, 0.0, 1e-2), (5, 10, 0.0, 0.6), (1, 10, 0.3 / tot, 0.0),
             (1, 10, 0.05 / tot, 0.0), (1, 2, 0.0, 0.0), (3, 6, 1e-2, 1e-12)]
    t = _tensor(tci, ctx, a)
    for chi_min, chi_max, target, smin in cases:
        u, s, vt, err = tci.trunc_svd(ctx, t, 1, chi_min, chi_max, target, smin)
        ru, rs, rvt, rerr = o_linalg.trunc_svd(a, 1, chi_min, chi_max, target, smin)
        assert s.to_numpy().shape == rs.shape, (chi_min, chi_max, target, smin)
        np.testing.assert_allclose(s.to_numpy(), rs, rtol=1e-12)
        assert abs(err - rerr) <= 1e-12 * max(1.0, rerr)
        assert u.shape == (6, rs.shape[0]) and vt.shape == (rs.shape[0], 8)


def test_dmrg_two_site_singlet(ctx, tci):
    e, _ = tci.dmrg(ctx, to_dev(heisenberg_mpo()), 2, 4, 2)
    assert abs(e[-1] + 0.75) < 1e-13


@pytest.mark.parametrize("n", [4, 8, 12])
def test_dmrg_matches_ed_without_truncation(ctx, tci, n):
    from test_oracle_dmrg import ed_ground
    e, terr = tci.dmrg(ctx, to_dev(heisenberg_mpo()), n, 2 ** (n // 2), 4)
    e0 = ed_ground(n)
    assert abs(e[-1] - e0) < 1e-10 * abs(e0)
    assert max(terr) < 1e-20


def test_truncated_dmrg_matches_oracle_sweeps(ctx, tci):
    n, chi = 14, 16
    e, terr = tci.dmrg(ctx, to_dev(heisenberg_mpo()), n, chi, 4)
    oe, oerr = o_dmrg.dmrg(heisenberg_mpo(), n, chi, 4)
    from test_oracle_dmrg import ed_ground
    e0 = ed_ground(n)
    assert e[-1] >= e0 - 1e-10
    assert abs(e[-1] - oe[-1]) < 1e-7 * abs(e0)
    assert max(terr) > 0.0


def test_dmrg_long_chain_bulk_energy_density(ctx, tci):
    """Open chains of 32 and 64 sites at chi_max 32 on the device: the bulk energy per site
    (E_64 - E_32) / 32 is within 3e-4 of 1/4 - ln 2 (the conformal 1/N term leaves 1.0e-4 in the
    difference, plus truncation), and each energy equals the oracle's sweeps."""
    e_inf = 0.25 - np.log(2.0)
    W = to_dev(heisenberg_mpo())
    e32, _ = tci.dmrg(ctx, W, 32, 32, 4)
    e64, _ = tci.dmrg(ctx, W, 64, 32, 4)
    bulk = (e64[-1] - e32[-1]) / 32
    assert 0.0 < bulk - e_inf < 3e-4, bulk
    oe64, _ = o_dmrg.dmrg(heisenberg_mpo(), 64, 32, 4)
    assert abs(e64[-1] - oe64[-1]) < 1e-8 * abs(oe64[-1])


def test_dmrg_split_precision_close_to_ed(ctx, tci):
    from test_oracle_dmrg import ed_ground
    ctx.set_precision("split_bf16")
    try:
        e, _ = tci.dmrg(ctx, to_dev(heisenberg_mpo()), 10, 32, 3)
    finally:
        ctx.set_precision("native")
    e0 = ed_ground(10)
    assert abs(e[-1] - e0) < 1e-6 * abs(e0)


@pytest.mark.parametrize("shape,k", [((1100, 1100), 1), ((5000, 20), 1), ((12, 3000), 1)])
def test_svd_long_rows_match_oracle(ctx, tci, shape, k):
    """Rows longer than 1024 take the scaled-rotation round (with and without QR preconditioning)."""
    a = random_tensor(shape, 31)
    u, s, vt = tci.svd(ctx, _tensor(tci, ctx, a), k)
    u, s, vt = u.to_numpy(), s.to_numpy(), vt.to_numpy()
    rs = o_linalg.svd(a, k)[1]
    np.testing.assert_allclose(s, rs, rtol=1e-12, atol=1e-12 * rs.max())
    _check_svd(a, k, u, s, vt, 1e-12)


def test_svd_rank_deficient_with_qr_preconditioning(ctx, tci):
    """Rank 5 of 60 columns (QR-preconditioned path): zero pivots in R, tiny singular values."""
    rng = np.random.default_rng(15)
    a = rng.standard_normal((80, 5)) @ rng.standard_normal((5, 60))
    u, s, vt = tci.svd(ctx, _tensor(tci, ctx, a), 1)
    s = s.to_numpy()
    np.testing.assert_allclose(s[:5], np.linalg.svd(a, compute_uv=False)[:5], rtol=1e-12)
    assert np.all(s[5:] < 1e-12 * s[0])
    _check_svd(a, 1, u.to_numpy(), s, vt.to_numpy(), 1e-12)
    ut, st, vtt, err = tci.trunc_svd(ctx, _tensor(tci, ctx, a), 1, 1, 60, 0.0, 1e-10)
    assert st.to_numpy().shape == (5,) and err < 1e-24                   # rule (a) drops the zero values
