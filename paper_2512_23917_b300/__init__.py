"""Python binding of ``libtci_b300.so`` (ctypes; argument marshalling only).

Every operation runs in the CUDA library; this module only turns torch
tensors into (pointer, shape, strides, dtype) tuples, passes the current
torch stream, and raises :class:`TciError` on a non-OK status.  There is no
fallback: if the shared library is missing this import fails.

Build the library with ``python -m paper_2512_23917_b300.build``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtci_b300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2512_23917_b300.build`")

lib = C.CDLL(LIB_PATH)

# ---------------------------------------------------------------- enums
F32, F64, C64, C128 = 0, 1, 2, 3
PREC_NATIVE, PREC_SPLIT_BF16, PREC_SPLIT_BF16_3 = 0, 1, 2
_PREC = {"native": PREC_NATIVE, "fp64": PREC_NATIVE, "split_bf16": PREC_SPLIT_BF16,
         "split_bf16_3": PREC_SPLIT_BF16_3}
STATUS = ["TCI_OK", "TCI_ERR_INVALID_ARG", "TCI_ERR_SHAPE", "TCI_ERR_LABEL", "TCI_ERR_DTYPE",
          "TCI_ERR_UNSUPPORTED", "TCI_ERR_ALLOC", "TCI_ERR_CUDA", "TCI_ERR_TIMEOUT",
          "TCI_ERR_INVALID_CONTEXT"]

_p = C.c_void_p
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_dp = C.POINTER(C.c_double)

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("tci_version", C.c_char_p, []),
    ("tci_status_string", C.c_char_p, [C.c_int]),
    ("tci_last_error", C.c_char_p, [_p]),
    ("tci_create_context", C.c_int, [C.POINTER(_p), C.c_int, _p]),
    ("tci_destroy_context", C.c_int, [C.POINTER(_p)]),
    ("tci_context_set_stream", C.c_int, [_p, _p]),
    ("tci_context_set_precision", C.c_int, [_p, C.c_int]),
    ("tci_context_get_precision", C.c_int, [_p, C.POINTER(C.c_int)]),
    ("tci_context_set_split_chunks", C.c_int, [_p, C.c_int, C.c_int]),
    ("tci_synchronize", C.c_int, [_p]),
    ("tci_tensor_wrap", C.c_int, [_p, C.c_int, C.c_int, _i64p, _i64p, _p, C.POINTER(_p)]),
    ("tci_allocate", C.c_int, [_p, C.c_int, C.c_int, _i64p, C.POINTER(_p)]),
    ("tci_zeros", C.c_int, [_p, C.c_int, C.c_int, _i64p, C.POINTER(_p)]),
    ("tci_copy", C.c_int, [_p, _p, C.POINTER(_p)]),
    ("tci_move", C.c_int, [_p, _p, C.POINTER(_p)]),
    ("tci_clear", C.c_int, [_p, _p]),
    ("tci_tensor_free", C.c_int, [C.POINTER(_p)]),
    ("tci_to_host", C.c_int, [_p, _p, _p]),
    ("tci_from_host", C.c_int, [_p, _p, _p]),
    ("tci_order", C.c_int, [_p, _p, C.POINTER(C.c_int)]),
    ("tci_shape", C.c_int, [_p, _p, _i64p]),
    ("tci_strides", C.c_int, [_p, _p, _i64p]),
    ("tci_size", C.c_int, [_p, _p, _i64p]),
    ("tci_size_bytes", C.c_int, [_p, _p, _i64p]),
    ("tci_get_dtype", C.c_int, [_p, _p, C.POINTER(C.c_int)]),
    ("tci_data", C.c_int, [_p, _p, C.POINTER(_p)]),
    ("tci_reshape", C.c_int, [_p, _p, C.c_int, _i64p]),
    ("tci_reshape_to", C.c_int, [_p, _p, C.c_int, _i64p, C.POINTER(_p)]),
    ("tci_transpose", C.c_int, [_p, _p, C.POINTER(C.c_int)]),
    ("tci_transpose_to", C.c_int, [_p, _p, C.POINTER(C.c_int), C.POINTER(_p)]),
    ("tci_contract", C.c_int, [_p, _p, C.c_char_p, _p, C.c_char_p, C.POINTER(_p), C.c_char_p]),
    ("tci_contract_l", C.c_int, [_p, _p, _i32p, _p, _i32p, C.POINTER(_p), _i32p, C.c_int]),
    ("tci_norm", C.c_int, [_p, _p, _dp]),
    ("tci_normalize", C.c_int, [_p, _p, _dp]),
    ("tci_scale", C.c_int, [_p, _p, C.c_double, C.c_double]),
    ("tci_linear_combine", C.c_int, [_p, C.c_int, C.POINTER(_p), _dp, C.POINTER(_p)]),
    ("tci_close", C.c_int, [_p, _p, _p, C.c_double, C.POINTER(C.c_int)]),
    ("tci_heff_plan_create", C.c_int, [_p, _p, _p, _p, C.POINTER(_p)]),
    ("tci_heff_plan_destroy", C.c_int, [C.POINTER(_p)]),
    ("tci_heff_apply", C.c_int, [_p, _p, _p]),
    ("tci_heff_apply_host", C.c_int, [_p, _p, _p]),
    ("tci_heff_apply_timed", C.c_int, [_p, _p, _p, C.POINTER(C.c_float)]),
    ("tci_heff_flops", C.c_double, [_p]),
    ("tci_heff_apply_noalloc", C.c_int, [_p, _p, _p, _p, _p, C.c_int64, C.c_int64, _p]),
    ("tci_bs_heff_plan_create", C.c_int, [_p, C.c_int, _i32p, _i64p, _i32p, _i32p, _p, _p, _p, C.POINTER(_p)]),
    ("tci_bs_plan_destroy", C.c_int, [C.POINTER(_p)]),
    ("tci_bs_heff_apply", C.c_int, [_p, _p, _p]),
    ("tci_bs_heff_flops", C.c_double, [_p]),
    ("tci_bs_psi_size", C.c_int64, [_p]),
    ("tci_tebd_plan_create", C.c_int, [_p, C.c_int, _i64p, C.POINTER(_p)]),
    ("tci_tebd_plan_destroy", C.c_int, [C.POINTER(_p)]),
    ("tci_tebd_apply", C.c_int, [_p, _p, _p, _p, _p]),
    ("tci_tebd_flops", C.c_double, [_p]),
    ("tci_tebd_apply_timed", C.c_int, [_p, _p, _p, _p, _p, C.POINTER(C.c_float)]),
    ("tci_tebd_tensor_flops", C.c_double, [_p]),
    ("tci_bs_heff_apply_timed", C.c_int, [_p, _p, _p, C.POINTER(C.c_float)]),
    ("tci_bs_tensor_flops", C.c_double, [_p]),
    ("tci_heff_autotune", C.c_int, [_p, _p, _p, C.c_int, C.POINTER(C.c_int)]),
    ("tci_bs_autotune", C.c_int, [_p, _p, C.c_int, C.POINTER(C.c_int)]),
    ("tci_tebd_autotune", C.c_int, [_p, _p, _p, _p, _p, C.c_int, C.POINTER(C.c_int)]),
    ("tci_lanczos", C.c_int, [_p, _p, C.c_int, C.c_int, _dp, _dp, _dp, C.POINTER(C.c_int), _p]),
    ("tci_heff_lanczos_stats", C.c_int, [_p, C.POINTER(C.c_int)]),
    ("tci_heff_set_lanczos_graphs", C.c_int, [_p, C.c_int]),
    ("tci_heff_lanczos_graph_info", C.c_int, [_p, _i64p]),
    ("tci_heff_set_lanczos_fused_dots", C.c_int, [_p, C.c_int]),
    ("tci_heff_set_lanczos_shadow_dots", C.c_int, [_p, C.c_int]),
    ("tci_bs_set_tile_n", C.c_int, [_p, C.c_int]),
    ("tci_bs_tile_n", C.c_int, [_p]),
    ("tci_bs_set_ww_variant", C.c_int, [_p, C.c_int]),
    ("tci_bs_ww_variant", C.c_int, [_p]),
    ("tci_tebd_set_tile_n", C.c_int, [_p, C.c_int]),
    ("tci_tebd_tile_n", C.c_int, [_p]),
    ("tci_heff_set_lanczos_reduced_terms", C.c_int, [_p, C.c_int]),
    ("tci_heff_plan_reload", C.c_int, [_p, _p, _p, _p, _p]),
    ("tci_heff_set_lanczos_arith", C.c_int, [_p, C.c_int]),
    ("tci_heff_plan_create2", C.c_int, [_p, _p, _p, _p, _p, C.POINTER(_p)]),
    ("tci_tebd_theta_batched", C.c_int, [_p, C.c_int, C.POINTER(_p), C.POINTER(_p), C.POINTER(_p), C.POINTER(_p)]),
    ("tci_heff_set_gram_schmidt", C.c_int, [_p, C.c_int]),
    ("tci_context_set_wait_limit", C.c_int, [_p, C.c_uint64]),
    ("tci_probe_fp64_rate", C.c_int, [_p, C.c_int, _dp]),
    ("tci_svd", C.c_int, [_p, _p, C.c_int, C.POINTER(_p), C.POINTER(_p), C.POINTER(_p)]),
    ("tci_trunc_svd", C.c_int, [_p, _p, C.c_int, C.POINTER(_p), C.POINTER(_p), C.POINTER(_p), _dp, C.c_int64,
                                C.c_int64, C.c_double, C.c_double]),
    ("tci_dmrg", C.c_int, [_p, _p, C.c_int, C.c_int64, C.c_int, C.c_int, C.c_double, _dp, _dp]),
    ("tci_bp", C.c_int, [_p, C.c_int, C.c_int, C.POINTER(C.c_int64), C.POINTER(_p), C.POINTER(_p), C.c_int, C.c_double,
                        C.POINTER(C.c_int), _dp]),
    ("tci_itebd", C.c_int, [_p, _p, C.c_double, _p, _p, _p, _p, C.c_int64, C.c_double, C.c_int, _dp, _dp]),
    ("tci_eye", C.c_int, [_p, C.c_int, C.c_int64, C.POINTER(_p)]),
    ("tci_fill", C.c_int, [_p, C.c_int, C.c_int, C.POINTER(C.c_int64), C.c_double, C.c_double, C.POINTER(_p)]),
    ("tci_cplx_conj", C.c_int, [_p, _p]),
    ("tci_cplx_conj_to", C.c_int, [_p, _p, C.POINTER(_p)]),
    ("tci_to_cplx", C.c_int, [_p, _p, C.POINTER(_p)]),
    ("tci_diag", C.c_int, [_p, _p]),
    ("tci_diag_to", C.c_int, [_p, _p, C.POINTER(_p)]),
    ("tci_heff_get_config", C.c_int, [_p, C.POINTER(C.c_int)]),
    ("tci_heff_set_config", C.c_int, [_p, C.POINTER(C.c_int)]),
]

for _name, _res, _args in SIGNATURES:
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class TciError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        self.status_name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{self.status_name}: {msg}")


def version() -> str:
    return lib.tci_version().decode()


def _check(status: int, ctx_handle=None):
    if status != 0:
        raise TciError(status, lib.tci_last_error(ctx_handle).decode(errors="replace"))


def _arr64(vals):
    vals = list(vals)
    return (C.c_int64 * max(1, len(vals)))(*vals)


_TORCH_DT = None


def _dtype_code(t) -> int:
    import torch
    m = {torch.float32: F32, torch.float64: F64, torch.complex64: C64, torch.complex128: C128}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


class Context:
    """TCI context bound to a CUDA device and the current torch stream."""

    def __init__(self, device: int = 0, stream=None, precision: str = "native"):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.handle = _p()
        _check(lib.tci_create_context(C.byref(self.handle), int(device), _p(int(stream))))
        self.device = device
        self.set_precision(precision)

    def set_precision(self, precision):
        code = _PREC[precision] if isinstance(precision, str) else int(precision)
        _check(lib.tci_context_set_precision(self.handle, code), self.handle)

    def set_split_chunks(self, chunk_k: int, xchunk_k: int):
        _check(lib.tci_context_set_split_chunks(self.handle, int(chunk_k), int(xchunk_k)), self.handle)

    def set_wait_limit(self, limit_ns: int):
        """Limit of the bounded device waits (ns; 0 = default 2 s)."""
        _check(lib.tci_context_set_wait_limit(self.handle, int(limit_ns)), self.handle)

    def probe_fp64_rate(self, iters: int = 20000) -> float:
        """Measured FP64 FMA rate of the device in GFLOP/s (a DFMA loop on every SM)."""
        g = C.c_double()
        _check(lib.tci_probe_fp64_rate(self.handle, int(iters), C.byref(g)), self.handle)
        return g.value

    def set_stream(self, stream: int):
        _check(lib.tci_context_set_stream(self.handle, _p(int(stream))), self.handle)

    def synchronize(self):
        _check(lib.tci_synchronize(self.handle), self.handle)

    def close(self):
        if self.handle:
            _check(lib.tci_destroy_context(C.byref(self.handle)))
            self.handle = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ tensors
    def wrap(self, t) -> "Tensor":
        """Borrowed TCI tensor view of a CUDA torch tensor (no copy)."""
        h = _p()
        _check(lib.tci_tensor_wrap(self.handle, _dtype_code(t), t.dim(), _arr64(t.shape), _arr64(t.stride()),
                                   _p(t.data_ptr()), C.byref(h)), self.handle)
        return Tensor(self, h, keepalive=t)


class Tensor:
    """Owner of a TCI tensor handle (borrowed view or library-owned storage)."""

    def __init__(self, ctx: Context, handle, keepalive=None):
        self.ctx = ctx
        self.handle = handle
        self._keep = keepalive

    @property
    def order(self) -> int:
        o = C.c_int()
        _check(lib.tci_order(self.ctx.handle, self.handle, C.byref(o)), self.ctx.handle)
        return o.value

    @property
    def shape(self):
        n = self.order
        a = (C.c_int64 * max(1, n))()
        _check(lib.tci_shape(self.ctx.handle, self.handle, a), self.ctx.handle)
        return tuple(a[:n])

    @property
    def strides(self):
        n = self.order
        a = (C.c_int64 * max(1, n))()
        _check(lib.tci_strides(self.ctx.handle, self.handle, a), self.ctx.handle)
        return tuple(a[:n])

    @property
    def dtype_code(self) -> int:
        d = C.c_int()
        _check(lib.tci_get_dtype(self.ctx.handle, self.handle, C.byref(d)), self.ctx.handle)
        return d.value

    def size(self) -> int:
        n = C.c_int64()
        _check(lib.tci_size(self.ctx.handle, self.handle, C.byref(n)), self.ctx.handle)
        return n.value

    def size_bytes(self) -> int:
        n = C.c_int64()
        _check(lib.tci_size_bytes(self.ctx.handle, self.handle, C.byref(n)), self.ctx.handle)
        return n.value

    def data_ptr(self) -> int:
        p = _p()
        _check(lib.tci_data(self.ctx.handle, self.handle, C.byref(p)), self.ctx.handle)
        return p.value or 0

    def to_numpy(self) -> np.ndarray:
        npdt = {F32: np.float32, F64: np.float64, C64: np.complex64, C128: np.complex128}[self.dtype_code]
        out = np.empty(self.shape, dtype=npdt)
        _check(lib.tci_to_host(self.ctx.handle, self.handle, _p(out.ctypes.data)), self.ctx.handle)
        return out

    def from_numpy(self, arr: np.ndarray):
        arr = np.ascontiguousarray(arr)
        _check(lib.tci_from_host(self.ctx.handle, self.handle, _p(arr.ctypes.data)), self.ctx.handle)

    def copy_from_host(self, address: int):
        """tci_from_host from a host buffer at ``address`` (e.g. pinned memory) holding size() elements."""
        _check(lib.tci_from_host(self.ctx.handle, self.handle, _p(int(address))), self.ctx.handle)

    def copy_to_host(self, address: int):
        """tci_to_host into a host buffer at ``address`` of size_bytes() bytes."""
        _check(lib.tci_to_host(self.ctx.handle, self.handle, _p(int(address))), self.ctx.handle)

    def reshape_(self, shape):
        _check(lib.tci_reshape(self.ctx.handle, self.handle, len(shape), _arr64(shape)), self.ctx.handle)
        return self

    def reshape(self, shape) -> "Tensor":
        h = _p()
        _check(lib.tci_reshape_to(self.ctx.handle, self.handle, len(shape), _arr64(shape), C.byref(h)),
               self.ctx.handle)
        return Tensor(self.ctx, h, keepalive=self)

    def transpose_(self, order):
        arr = (C.c_int * max(1, len(order)))(*order)
        _check(lib.tci_transpose(self.ctx.handle, self.handle, arr), self.ctx.handle)
        return self

    def transpose(self, order) -> "Tensor":
        arr = (C.c_int * max(1, len(order)))(*order)
        h = _p()
        _check(lib.tci_transpose_to(self.ctx.handle, self.handle, arr, C.byref(h)), self.ctx.handle)
        return Tensor(self.ctx, h)

    def copy(self) -> "Tensor":
        h = _p()
        _check(lib.tci_copy(self.ctx.handle, self.handle, C.byref(h)), self.ctx.handle)
        return Tensor(self.ctx, h)

    def move(self) -> "Tensor":
        h = _p()
        _check(lib.tci_move(self.ctx.handle, self.handle, C.byref(h)), self.ctx.handle)
        return Tensor(self.ctx, h, keepalive=self._keep)

    def clear(self):
        _check(lib.tci_clear(self.ctx.handle, self.handle), self.ctx.handle)

    def norm(self) -> float:
        v = C.c_double()
        _check(lib.tci_norm(self.ctx.handle, self.handle, C.byref(v)), self.ctx.handle)
        return v.value

    def normalize_(self) -> float:
        v = C.c_double()
        _check(lib.tci_normalize(self.ctx.handle, self.handle, C.byref(v)), self.ctx.handle)
        return v.value

    def scale_(self, s):
        s = complex(s)
        _check(lib.tci_scale(self.ctx.handle, self.handle, s.real, s.imag), self.ctx.handle)
        return self

    def cplx_conj_(self):
        _check(lib.tci_cplx_conj(self.ctx.handle, self.handle), self.ctx.handle)
        return self

    def cplx_conj(self) -> "Tensor":
        h = _p()
        _check(lib.tci_cplx_conj_to(self.ctx.handle, self.handle, C.byref(h)), self.ctx.handle)
        return Tensor(self.ctx, h)

    def to_cplx(self) -> "Tensor":
        h = _p()
        _check(lib.tci_to_cplx(self.ctx.handle, self.handle, C.byref(h)), self.ctx.handle)
        return Tensor(self.ctx, h)

    def diag_(self):
        _check(lib.tci_diag(self.ctx.handle, self.handle), self.ctx.handle)
        return self

    def diag(self) -> "Tensor":
        h = _p()
        _check(lib.tci_diag_to(self.ctx.handle, self.handle, C.byref(h)), self.ctx.handle)
        return Tensor(self.ctx, h)

    def free(self):
        if self.handle:
            _check(lib.tci_tensor_free(C.byref(self.handle)))
            self.handle = _p()

    def __del__(self):
        try:
            if self.handle and self.ctx.handle:
                lib.tci_tensor_free(C.byref(self.handle))
        except Exception:
            pass


def svd(ctx: Context, t: Tensor, num_of_bds_as_row: int):
    """TCI svd of a tensor handle: (u, s, v_dag) as new Tensors."""
    hu, hs, hv = _p(), _p(), _p()
    _check(lib.tci_svd(ctx.handle, t.handle, int(num_of_bds_as_row), C.byref(hu), C.byref(hs), C.byref(hv)),
           ctx.handle)
    return Tensor(ctx, hu), Tensor(ctx, hs), Tensor(ctx, hv)


def trunc_svd(ctx: Context, t: Tensor, num_of_bds_as_row: int, chi_min: int, chi_max: int,
              target_trunc_err: float = 0.0, s_min: float = 0.0):
    """TCI trunc_svd: (u, s, v_dag, trunc_err)."""
    hu, hs, hv = _p(), _p(), _p()
    err = C.c_double()
    _check(lib.tci_trunc_svd(ctx.handle, t.handle, int(num_of_bds_as_row), C.byref(hu), C.byref(hs), C.byref(hv),
                             C.byref(err), int(chi_min), int(chi_max), float(target_trunc_err), float(s_min)),
           ctx.handle)
    return Tensor(ctx, hu), Tensor(ctx, hs), Tensor(ctx, hv), err.value


def dmrg(ctx: Context, W, nsites: int, chi_max: int, nsweeps: int, lanczos_steps: int = 20, s_min: float = 1e-12):
    """Two-site DMRG on the device (W: CUDA float64 [Dw, Dw, 2, 2]); returns (energies, max truncation errors)."""
    e = (C.c_double * nsweeps)()
    te = (C.c_double * nsweeps)()
    tw = ctx.wrap(W)
    _check(lib.tci_dmrg(ctx.handle, tw.handle, int(nsites), int(chi_max), int(nsweeps), int(lanczos_steps),
                        float(s_min), e, te), ctx.handle)
    return list(e), list(te)


def itebd(ctx: Context, h, dt: float, gammas, lambdas, chi: int, niters: int, s_min: float = 1e-10):
    """App. A iTEBD on the device.  h: numpy [4, 4]; gammas / lambdas: numpy arrays of the unit cell.

    Returns (energies, truncation errors, final gammas, final lambdas) as numpy arrays.
    """
    ht = allocate(ctx, [4, 4], F64)
    ht.from_numpy(np.asarray(h, dtype=np.float64).reshape(4, 4))
    cell = []
    for a in list(gammas) + list(lambdas):
        t = allocate(ctx, np.shape(a), F64)
        t.from_numpy(np.asarray(a, dtype=np.float64))
        cell.append(t)
    e = (C.c_double * max(1, niters))()
    te = (C.c_double * max(1, niters))()
    _check(lib.tci_itebd(ctx.handle, ht.handle, float(dt), cell[0].handle, cell[1].handle, cell[2].handle,
                         cell[3].handle, int(chi), float(s_min), int(niters), e, te), ctx.handle)
    out = [t.to_numpy() for t in cell]
    return list(e[:niters]), list(te[:niters]), out[:2], out[2:]


def bp(ctx: Context, n: int, edges, sites, messages, niters: int, tol: float = 0.0):
    """App. B belief propagation on the device.  sites / messages: numpy arrays (messages per edge e:
    2e = u -> v, 2e + 1 = v -> u).  Returns (messages as numpy arrays, residual per iteration)."""
    st = []
    for a in sites:
        t = allocate(ctx, np.shape(a), F64)
        t.from_numpy(np.asarray(a, dtype=np.float64))
        st.append(t)
    mt = []
    for a in messages:
        t = allocate(ctx, np.shape(a), F64)
        t.from_numpy(np.asarray(a, dtype=np.float64))
        mt.append(t)
    ed = (C.c_int64 * max(1, 2 * len(edges)))(*[int(x) for e in edges for x in e])
    sh = (_p * max(1, len(st)))(*[t.handle for t in st])
    mh = (_p * max(1, len(mt)))(*[t.handle for t in mt])
    res = (C.c_double * max(1, niters))()
    done = C.c_int()
    _check(lib.tci_bp(ctx.handle, int(n), len(edges), ed, sh, mh, int(niters), float(tol), C.byref(done), res),
           ctx.handle)
    return [t.to_numpy() for t in mt], list(res[:done.value])


def tebd_theta_batched(ctx: Context, A, B, G):
    """Batched TEBD theta on lists of CUDA complex64 torch tensors; returns new TCI Tensors theta_i."""
    ta = [ctx.wrap(a) for a in A]
    tb = [ctx.wrap(b) for b in B]
    tg = [ctx.wrap(g) for g in G]
    n = len(ta)
    ha = (_p * max(1, n))(*[t.handle for t in ta])
    hb = (_p * max(1, n))(*[t.handle for t in tb])
    hg = (_p * max(1, n))(*[t.handle for t in tg])
    ht = (_p * max(1, n))()
    _check(lib.tci_tebd_theta_batched(ctx.handle, n, ha, hb, hg, ht), ctx.handle)
    return [Tensor(ctx, ht[i]) for i in range(n)]


def eye(ctx: Context, n: int, dtype: int = F64) -> Tensor:
    h = _p()
    _check(lib.tci_eye(ctx.handle, dtype, int(n), C.byref(h)), ctx.handle)
    return Tensor(ctx, h)


def fill(ctx: Context, shape, value, dtype: int = F64) -> Tensor:
    h = _p()
    v = complex(value)
    _check(lib.tci_fill(ctx.handle, dtype, len(shape), _arr64(shape), v.real, v.imag, C.byref(h)), ctx.handle)
    return Tensor(ctx, h)


def allocate(ctx: Context, shape, dtype: int = F64, zero: bool = False) -> Tensor:
    h = _p()
    fn = lib.tci_zeros if zero else lib.tci_allocate
    _check(fn(ctx.handle, dtype, len(shape), _arr64(shape), C.byref(h)), ctx.handle)
    return Tensor(ctx, h)


def contract_into(ctx: Context, a: Tensor, la, b: Tensor, lb, c, lc) -> Tensor:
    """TCI contract with handles; ``c`` is a Tensor (written / re-allocated) or None (new owned)."""
    h = c.handle if c is not None else _p()
    if isinstance(la, str):
        _check(lib.tci_contract(ctx.handle, a.handle, la.encode(), b.handle, lb.encode(), C.byref(h),
                                lc.encode()), ctx.handle)
    else:
        ia = (C.c_int32 * max(1, len(la)))(*la)
        ib = (C.c_int32 * max(1, len(lb)))(*lb)
        ic = (C.c_int32 * max(1, len(lc)))(*lc)
        _check(lib.tci_contract_l(ctx.handle, a.handle, ia, b.handle, ib, C.byref(h), ic, len(lc)), ctx.handle)
    if c is not None:
        c.handle = h
        return c
    return Tensor(ctx, h)


def contract(ctx: Context, a, la, b, lb, lc, out=None):
    """C = contract(a, la, b, lb, lc) on torch CUDA tensors (string or int labels).

    ``out`` (optional) is a torch tensor of the output shape that receives
    the result; otherwise one is allocated.  Returns the torch output.
    """
    import torch
    la_l, lb_l, lc_l = list(la), list(lb), list(lc)
    if out is None:
        dims = dict(zip(la_l, a.shape))
        dims.update(zip(lb_l, b.shape))
        shape = [dims[l] for l in lc_l] if all(l in dims for l in lc_l) else [0]
        out = torch.empty(shape, dtype=a.dtype, device=a.device)
    ta, tb, tc = ctx.wrap(a), ctx.wrap(b), ctx.wrap(out)
    contract_into(ctx, ta, la, tb, lb, tc, lc)
    return out


def linear_combine(ctx: Context, tensors, coefs, out):
    keep = [ctx.wrap(t) for t in tensors]
    hs = (_p * len(tensors))(*[k.handle for k in keep])
    co = (C.c_double * len(tensors))(*coefs) if coefs is not None else None
    to = ctx.wrap(out)
    h = to.handle
    _check(lib.tci_linear_combine(ctx.handle, len(tensors), hs, co, C.byref(h)), ctx.handle)
    return out


def close(ctx: Context, a, b, eps: float) -> bool:
    r = C.c_int()
    ta, tb = ctx.wrap(a), ctx.wrap(b)
    _check(lib.tci_close(ctx.handle, ta.handle, tb.handle, float(eps), C.byref(r)), ctx.handle)
    return bool(r.value)


class HeffPlan:
    """Two-site H_eff plan (see include/tci_b300.h, tci_heff_plan_create)."""

    def __init__(self, ctx: Context, L, W, R, precision=None, W2=None):
        """``W2`` (optional): a different MPO tensor for the right site (tci_heff_plan_create2)."""
        if precision is not None:
            ctx.set_precision(precision)
        self.ctx = ctx
        self.handle = _p()
        self.chiL, self.chiR = L.shape[0], R.shape[0]
        tl, tw, tr = ctx.wrap(L), ctx.wrap(W), ctx.wrap(R)
        if W2 is None:
            _check(lib.tci_heff_plan_create(ctx.handle, tl.handle, tw.handle, tr.handle, C.byref(self.handle)),
                   ctx.handle)
        else:
            tw2 = ctx.wrap(W2)
            _check(lib.tci_heff_plan_create2(ctx.handle, tl.handle, tw.handle, tw2.handle, tr.handle,
                                             C.byref(self.handle)), ctx.handle)
        self._psi_wrap = {}

    @property
    def flops(self) -> float:
        return lib.tci_heff_flops(self.handle)

    def apply(self, psi, out):
        tp, to = self.ctx.wrap(psi), self.ctx.wrap(out)
        _check(lib.tci_heff_apply(self.handle, tp.handle, to.handle), self.ctx.handle)
        return out

    def apply_timed(self, psi, out):
        """Apply and return the four stage durations in ms (split, GEMM1, W.W, GEMM2)."""
        ms = (C.c_float * 4)()
        tp, to = self.ctx.wrap(psi), self.ctx.wrap(out)
        _check(lib.tci_heff_apply_timed(self.handle, tp.handle, to.handle, ms), self.ctx.handle)
        return list(ms)

    def autotune(self, psi, out, max_chunk_k: int = 256):
        """Tune the split GEMM configuration on these operands; returns (chunk_k, xchunk_k, raster)."""
        ch = (C.c_int * 3)()
        tp, to = self.ctx.wrap(psi), self.ctx.wrap(out)
        _check(lib.tci_heff_autotune(self.handle, tp.handle, to.handle, int(max_chunk_k), ch), self.ctx.handle)
        return tuple(ch)

    def get_config(self):
        """(chunk_k, xchunk_k, raster, W.W a' per thread) of a split-BF16 plan."""
        cfg = (C.c_int * 4)()
        _check(lib.tci_heff_get_config(self.handle, cfg), self.ctx.handle)
        return tuple(cfg)

    def set_config(self, chunk_k: int, xchunk_k: int, raster: int, ww_na: int):
        cfg = (C.c_int * 4)(int(chunk_k), int(xchunk_k), int(raster), int(ww_na))
        _check(lib.tci_heff_set_config(self.handle, cfg), self.ctx.handle)

    def apply_host(self, psi_host: np.ndarray, out_host: np.ndarray):
        assert psi_host.dtype == np.float64 and out_host.dtype == np.float64
        assert psi_host.flags.c_contiguous and out_host.flags.c_contiguous
        _check(lib.tci_heff_apply_host(self.handle, _p(psi_host.ctypes.data), _p(out_host.ctypes.data)),
               self.ctx.handle)
        return out_host

    LANCZOS_ARITH = {"auto": 0, "f64": 1, "df32": 2}

    def set_lanczos_arith(self, arith: str):
        """Vector arithmetic of lanczos(): "auto", "f64" or "df32" (double-float FP32 pairs)."""
        _check(lib.tci_heff_set_lanczos_arith(self.handle, self.LANCZOS_ARITH[arith]), self.ctx.handle)

    GRAM_SCHMIDT = {"dgks": 0, "twice": 1}

    def set_gram_schmidt(self, mode: str):
        """Re-orthogonalisation of lanczos(): "dgks" (second pass where the first cancelled) or "twice"."""
        _check(lib.tci_heff_set_gram_schmidt(self.handle, self.GRAM_SCHMIDT[mode]), self.ctx.handle)

    def lanczos(self, psi0, nsteps: int, reorth: bool = True, x=None):
        ritz = C.c_double()
        alpha = (C.c_double * nsteps)()
        beta = (C.c_double * nsteps)()
        k = C.c_int()
        tp = self.ctx.wrap(psi0)
        tx = self.ctx.wrap(x) if x is not None else None
        _check(lib.tci_lanczos(self.handle, tp.handle, int(nsteps), int(bool(reorth)), C.byref(ritz), alpha, beta,
                               C.byref(k), tx.handle if tx is not None else None), self.ctx.handle)
        return {"theta": ritz.value, "alpha": np.array(alpha[:k.value]), "beta": np.array(beta[:k.value]),
                "steps": k.value}

    def set_lanczos_graphs(self, enable: bool):
        """Replay repeated lanczos() calls from a captured CUDA graph (default on, real plans;
        complex plans run eagerly)."""
        _check(lib.tci_heff_set_lanczos_graphs(self.handle, int(bool(enable))), self.ctx.handle)

    def reload(self, L, W, R, W2=None):
        """New environments / MPO tensors of the same shapes (torch CUDA tensors) for this plan."""
        tl, tw, tr = self.ctx.wrap(L), self.ctx.wrap(W), self.ctx.wrap(R)
        tw2 = self.ctx.wrap(W2) if W2 is not None else None
        _check(lib.tci_heff_plan_reload(self.handle, tl.handle, tw.handle, tw2.handle if tw2 is not None else None,
                                        tr.handle), self.ctx.handle)
        self._keep = (L, W, R, W2)

    def set_lanczos_fused_dots(self, enable: bool):
        """Form the first projection's dots in the matvec's GEMM2 epilogue (split plans; off by default:
        slower on B300 than the separate pass)."""
        _check(lib.tci_heff_set_lanczos_fused_dots(self.handle, int(bool(enable))), self.ctx.handle)

    def set_lanczos_shadow_dots(self, enable: bool):
        """Double-float Gram-Schmidt dots on the FP32 pipes (split plans, FP64 vectors; off by default:
        the Lanczos dot products are FP64)."""
        _check(lib.tci_heff_set_lanczos_shadow_dots(self.handle, int(bool(enable))), self.ctx.handle)

    def set_lanczos_reduced_terms(self, enable: bool):
        """Allow (default) or forbid the FP32 / double-float evaluation of small update terms."""
        _check(lib.tci_heff_set_lanczos_reduced_terms(self.handle, int(bool(enable))), self.ctx.handle)

    def lanczos_stats(self):
        """Counters of the last lanczos(): steps, repeated projections, update passes with FP32 /
        double-float small terms, second projections folded into the next-vector pass."""
        st = (C.c_int * 5)()
        _check(lib.tci_heff_lanczos_stats(self.handle, st), self.ctx.handle)
        return {"steps": st[0], "second_passes": st[1], "f32_term_passes": st[2], "df_term_passes": st[3],
                "fused_pass3": st[4]}

    def lanczos_graph_info(self):
        """Graph replay state: enabled (False after a capture failed), whether the last lanczos()
        ran as one graph launch, and the number of graph launches of this plan."""
        info = (C.c_int64 * 3)()
        _check(lib.tci_heff_lanczos_graph_info(self.handle, info), self.ctx.handle)
        return {"enabled": bool(info[0]), "last_from_graph": bool(info[1]), "graph_launches": int(info[2])}

    def close(self):
        if self.handle:
            _check(lib.tci_heff_plan_destroy(C.byref(self.handle)))
            self.handle = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BsHeffPlan:
    """U(1) block-sparse H_eff plan (see include/tci_b300.h, tci_bs_heff_plan_create).

    ``sector_charge``/``sector_dim`` list the bond sectors; ``L_packed`` and
    ``R_packed`` are CUDA float32 tensors holding the blocks in the canonical
    packed order; ``W`` a CUDA float64 [5,5,2,2] tensor.
    """

    def __init__(self, ctx: Context, sector_charge, sector_dim, phys_charge, mpo_charge, L_packed, R_packed, W,
                 precision="split_bf16"):
        ctx.set_precision(precision)
        self.ctx = ctx
        self.handle = _p()
        n = len(sector_charge)
        qc = (C.c_int32 * n)(*[int(q) for q in sector_charge])
        qd = (C.c_int64 * n)(*[int(d) for d in sector_dim])
        pc = (C.c_int32 * len(phys_charge))(*[int(c) for c in phys_charge])
        mc = (C.c_int32 * len(mpo_charge))(*[int(c) for c in mpo_charge])
        _check(lib.tci_bs_heff_plan_create(ctx.handle, n, qc, qd, pc, mc, _p(L_packed.data_ptr()),
                                           _p(R_packed.data_ptr()), _p(W.data_ptr()), C.byref(self.handle)),
               ctx.handle)

    @property
    def flops(self) -> float:
        return lib.tci_bs_heff_flops(self.handle)

    @property
    def psi_size(self) -> int:
        return lib.tci_bs_psi_size(self.handle)

    @property
    def tensor_flops(self) -> float:
        return lib.tci_bs_tensor_flops(self.handle)

    def autotune(self, psi_packed, max_chunk_k: int = 256):
        """Tune the grouped GEMMs; returns (chunk_k, xchunk_k, raster); the tile width is tile_n."""
        ch = (C.c_int * 3)()
        _check(lib.tci_bs_autotune(self.handle, _p(psi_packed.data_ptr()), int(max_chunk_k), ch), self.ctx.handle)
        return tuple(ch)

    @property
    def tile_n(self) -> int:
        return lib.tci_bs_tile_n(self.handle)

    def set_tile_n(self, bn: int):
        _check(lib.tci_bs_set_tile_n(self.handle, int(bn)), self.ctx.handle)

    @property
    def ww_variant(self) -> int:
        return lib.tci_bs_ww_variant(self.handle)

    def set_ww_variant(self, variant: int):
        _check(lib.tci_bs_set_ww_variant(self.handle, int(variant)), self.ctx.handle)

    def apply_timed(self, psi_packed, out_packed):
        ms = (C.c_float * 4)()
        _check(lib.tci_bs_heff_apply_timed(self.handle, _p(psi_packed.data_ptr()), _p(out_packed.data_ptr()), ms),
               self.ctx.handle)
        return list(ms)

    def apply(self, psi_packed, out_packed):
        _check(lib.tci_bs_heff_apply(self.handle, _p(psi_packed.data_ptr()), _p(out_packed.data_ptr())),
               self.ctx.handle)
        return out_packed

    def close(self):
        if self.handle:
            _check(lib.tci_bs_plan_destroy(C.byref(self.handle)))
            self.handle = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_blocks(blocks: dict, keys) -> np.ndarray:
    """Concatenate blocks (row-major) in the given key order into one float32 vector."""
    if not keys:
        return np.zeros(0, dtype=np.float32)
    return np.concatenate([np.ascontiguousarray(blocks[k], dtype=np.float32).ravel() for k in keys])


def unpack_blocks(vec: np.ndarray, keys, shapes) -> dict:
    out, off = {}, 0
    for k in keys:
        r, c = shapes[k]
        out[k] = vec[off:off + r * c].reshape(r, c)
        off += r * c
    return out


class TebdPlan:
    """Batched TEBD theta plan (see include/tci_b300.h, tci_tebd_plan_create)."""

    def __init__(self, ctx: Context, chis, precision="split_bf16"):
        ctx.set_precision(precision)
        self.ctx = ctx
        self.chis = [int(c) for c in chis]
        self.handle = _p()
        arr = (C.c_int64 * len(self.chis))(*self.chis)
        _check(lib.tci_tebd_plan_create(ctx.handle, len(self.chis), arr, C.byref(self.handle)), ctx.handle)

    @property
    def flops(self) -> float:
        return lib.tci_tebd_flops(self.handle)

    @property
    def tensor_flops(self) -> float:
        return lib.tci_tebd_tensor_flops(self.handle)

    @property
    def tile_n(self) -> int:
        return lib.tci_tebd_tile_n(self.handle)

    def set_tile_n(self, bn: int):
        _check(lib.tci_tebd_set_tile_n(self.handle, int(bn)), self.ctx.handle)

    def autotune(self, A_packed, B_packed, G_packed, theta_packed, max_chunk_k: int = 256):
        ch = (C.c_int * 3)()
        _check(lib.tci_tebd_autotune(self.handle, _p(A_packed.data_ptr()), _p(B_packed.data_ptr()),
                                     _p(G_packed.data_ptr()), _p(theta_packed.data_ptr()), int(max_chunk_k), ch),
               self.ctx.handle)
        return tuple(ch)

    def apply_timed(self, A_packed, B_packed, G_packed, theta_packed):
        ms = (C.c_float * 3)()
        _check(lib.tci_tebd_apply_timed(self.handle, _p(A_packed.data_ptr()), _p(B_packed.data_ptr()),
                                        _p(G_packed.data_ptr()), _p(theta_packed.data_ptr()), ms), self.ctx.handle)
        return list(ms)

    def apply(self, A_packed, B_packed, G_packed, theta_packed):
        _check(lib.tci_tebd_apply(self.handle, _p(A_packed.data_ptr()), _p(B_packed.data_ptr()),
                                  _p(G_packed.data_ptr()), _p(theta_packed.data_ptr())), self.ctx.handle)
        return theta_packed

    def close(self):
        if self.handle:
            _check(lib.tci_tebd_plan_destroy(C.byref(self.handle)))
            self.handle = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
