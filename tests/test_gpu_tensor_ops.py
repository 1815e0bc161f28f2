"""Device eye / fill / cplx_conj / to_cplx / diag (App. C.2) against the oracle."""
import numpy as np
import pytest

from oracle import tensor_ops as o

pytestmark = pytest.mark.gpu

DT = {"f32": (0, np.float32), "f64": (1, np.float64), "c64": (2, np.complex64), "c128": (3, np.complex128)}


@pytest.mark.parametrize("dt", list(DT))
@pytest.mark.parametrize("n", [0, 1, 3, 257])
def test_eye(ctx, tci, dt, n):
    code, npdt = DT[dt]
    t = tci.eye(ctx, n, code)
    assert t.shape == (n, n)
    np.testing.assert_array_equal(t.to_numpy(), o.eye(n, npdt))


@pytest.mark.parametrize("dt", list(DT))
def test_fill(ctx, tci, dt):
    code, npdt = DT[dt]
    v = 2.0 if code < 2 else 2.0 - 0.5j
    t = tci.fill(ctx, [3, 2, 4], v, code)
    np.testing.assert_array_equal(t.to_numpy(), o.fill([3, 2, 4], v, npdt))
    assert tci.fill(ctx, [0, 5], v, code).size() == 0


@pytest.mark.parametrize("dt", list(DT))
def test_cplx_conj_in_and_out_of_place_on_a_lazy_view(ctx, tci, dt):
    code, npdt = DT[dt]
    rng = np.random.default_rng(5)
    a = rng.standard_normal((3, 2, 4))
    if code >= 2:
        a = a + 1j * rng.standard_normal((3, 2, 4))
    a = a.astype(npdt)
    t = tci.allocate(ctx, a.shape, code)
    t.from_numpy(a)
    t.transpose_([2, 0, 1])                     # lazy permutation: strided input
    ref = o.cplx_conj(np.transpose(a, (2, 0, 1)))
    np.testing.assert_array_equal(t.cplx_conj().to_numpy(), ref)
    t.cplx_conj_()
    np.testing.assert_array_equal(t.to_numpy(), ref)


@pytest.mark.parametrize("dt", ["f32", "f64", "c128"])
def test_to_cplx(ctx, tci, dt):
    code, npdt = DT[dt]
    a = np.arange(12, dtype=np.float64).reshape(3, 4).astype(npdt)
    t = tci.allocate(ctx, a.shape, code)
    t.from_numpy(a)
    z = t.to_cplx()
    ref = o.to_cplx(a)
    assert z.to_numpy().dtype == ref.dtype
    np.testing.assert_array_equal(z.to_numpy(), ref)


@pytest.mark.parametrize("dt", list(DT))
def test_diag_paper_roundtrip_and_rectangular(ctx, tci, dt):
    code, npdt = DT[dt]
    e = tci.eye(ctx, 3, code)
    e.diag_()
    assert e.order == 1
    e.diag_()
    np.testing.assert_array_equal(e.to_numpy(), o.eye(3, npdt))
    rng = np.random.default_rng(6)
    r = rng.standard_normal((5, 7)).astype(npdt)
    t = tci.allocate(ctx, r.shape, code)
    t.from_numpy(r)
    np.testing.assert_array_equal(t.diag().to_numpy(), o.diag(r))
    t.transpose_([1, 0])                        # diag of a lazy transpose
    np.testing.assert_array_equal(t.diag().to_numpy(), o.diag(r.T))
    v = rng.standard_normal(6).astype(npdt)
    tv = tci.allocate(ctx, v.shape, code)
    tv.from_numpy(v)
    np.testing.assert_array_equal(tv.diag().to_numpy(), o.diag(v))


def test_diag_rejects_other_orders(ctx, tci):
    t = tci.allocate(ctx, [2, 2, 2], 1)
    with pytest.raises(tci.TciError):
        t.diag()
