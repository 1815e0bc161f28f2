// TCI construction and elementwise functions of App. C.2 on the device:
// eye, fill ("Tensor construction"), cplx_conj and to_cplx ("Tensor
// manipulation"), diag ("Tensor linear algebra").  Inputs may carry lazy
// (strided) layouts; outputs are new owned row-major tensors, and the
// in-place forms replace the tensor's storage.
#include "tci_internal.cuh"

namespace {

template <typename T>
__device__ __forceinline__ T make_val(double re, double im);
template <> __device__ __forceinline__ float make_val<float>(double re, double) { return (float)re; }
template <> __device__ __forceinline__ double make_val<double>(double re, double) { return re; }
template <> __device__ __forceinline__ float2 make_val<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> __device__ __forceinline__ double2 make_val<double2>(double re, double im) { return make_double2(re, im); }

template <typename T>
__global__ void k_fill(T* __restrict__ x, int64_t n, double re, double im) {
  const T v = make_val<T>(re, im);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

// out (n x n, zeroed) gets v[i * stride] on its diagonal
template <typename T>
__global__ void k_diag_promote(const T* __restrict__ v, int64_t stride, T* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i * n + i] = v[i * stride];
}

// out[i] = a[i * (s0 + s1)], i < m
template <typename T>
__global__ void k_diag_extract(const T* __restrict__ a, int64_t step, T* __restrict__ out, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i * step];
}

template <typename C>
__global__ void k_conj(C* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i].y = -x[i].y;
}

template <typename R, typename C>
__global__ void k_to_cplx(const R* __restrict__ in, C* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    C c;
    c.x = in[i];
    c.y = 0;
    out[i] = c;
  }
}

int grid_for(tci_context ctx, int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)ctx->num_sms * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// Calls f(T{}) with T the element type of dt.
template <typename F>
tci_status dispatch(tci_context ctx, tci_dtype dt, F f) {
  switch (dt) {
    case TCI_F32: f(float()); break;
    case TCI_F64: f(double()); break;
    case TCI_C64: f(float2()); break;
    case TCI_C128: f(double2()); break;
    default: return tci_fail(ctx, TCI_ERR_DTYPE, "unknown dtype");
  }
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

template <typename T>
__global__ void k_eye_diag(T* __restrict__ out, int64_t n) {
  const T one = make_val<T>(1.0, 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i * n + i] = one;
}

// Replace t's metadata and storage by those of src (src is consumed).
void adopt(tci_context ctx, tci_tensor t, tci_tensor src) {
  if (t->alloc) {
    cudaStreamSynchronize(ctx->stream);
    tci_dev_free(t->alloc);
  }
  t->dtype = src->dtype;
  t->order = src->order;
  for (int i = 0; i < src->order; ++i) {
    t->shape[i] = src->shape[i];
    t->strides[i] = src->strides[i];
  }
  t->data = src->data;
  t->alloc = src->alloc;
  src->alloc = nullptr;
  tci_tensor tmp = src;
  tci_tensor_free(&tmp);
}

}  // namespace

extern "C" tci_status tci_eye(tci_context ctx, tci_dtype dtype, int64_t n, tci_tensor* out) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "eye");
  if (n < 0) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "eye: negative dimension");
  const int64_t shape[2] = {n, n};
  TCI_TRY(tci_zeros(ctx, dtype, 2, shape, out));
  if (n == 0) return TCI_OK;
  tci_tensor t = *out;
  return dispatch(ctx, dtype, [&](auto tag) {
    using T = decltype(tag);
    k_eye_diag<T><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((T*)t->data, n);
  });
}

extern "C" tci_status tci_fill(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape, double re, double im,
                               tci_tensor* out) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "fill");
  TCI_TRY(tci_allocate(ctx, dtype, order, shape, out));
  tci_tensor t = *out;
  const int64_t n = tci_numel(t);
  if (n == 0) return TCI_OK;
  return dispatch(ctx, dtype, [&](auto tag) {
    using T = decltype(tag);
    k_fill<T><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((T*)t->data, n, re, im);
  });
}

extern "C" tci_status tci_cplx_conj_to(tci_context ctx, tci_tensor in, tci_tensor* out) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(in)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "cplx_conj: invalid tensor");
  TciVerboseScope vs(ctx, "cplx_conj");
  TCI_TRY(tci_copy(ctx, in, out));
  const int64_t n = tci_numel(*out);
  if (n == 0) return TCI_OK;
  if (in->dtype == TCI_C64) k_conj<float2><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((float2*)(*out)->data, n);
  else if (in->dtype == TCI_C128) k_conj<double2><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((double2*)(*out)->data, n);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

extern "C" tci_status tci_cplx_conj(tci_context ctx, tci_tensor t) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "cplx_conj: invalid tensor");
  if (t->dtype != TCI_C64 && t->dtype != TCI_C128) return TCI_OK;   // real: no change
  TciVerboseScope vs(ctx, "cplx_conj");
  TCI_TRY(tci_materialise(ctx, t));
  const int64_t n = tci_numel(t);
  if (n == 0) return TCI_OK;
  if (t->dtype == TCI_C64) k_conj<float2><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((float2*)t->data, n);
  else k_conj<double2><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((double2*)t->data, n);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

extern "C" tci_status tci_to_cplx(tci_context ctx, tci_tensor in, tci_tensor* out) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(in)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "to_cplx: invalid tensor");
  TciVerboseScope vs(ctx, "to_cplx");
  if (in->dtype == TCI_C64 || in->dtype == TCI_C128) return tci_copy(ctx, in, out);
  tci_tensor src = in;
  tci_tensor tmp = nullptr;
  if (!tci_is_rowmajor(in)) {
    TCI_TRY(tci_copy(ctx, in, &tmp));
    src = tmp;
  }
  const tci_dtype cd = in->dtype == TCI_F32 ? TCI_C64 : TCI_C128;
  tci_status s = tci_allocate(ctx, cd, in->order, in->shape, out);
  const int64_t n = tci_numel(in);
  if (s == TCI_OK && n > 0) {
    if (cd == TCI_C64)
      k_to_cplx<float, float2><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((const float*)src->data, (float2*)(*out)->data, n);
    else
      k_to_cplx<double, double2><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((const double*)src->data, (double2*)(*out)->data, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = tci_cuda_fail(ctx, e, "to_cplx");
  }
  if (tmp) {
    cudaStreamSynchronize(ctx->stream);
    tci_tensor_free(&tmp);
  }
  return s;
}

extern "C" tci_status tci_diag_to(tci_context ctx, tci_tensor in, tci_tensor* out) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(in)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "diag: invalid tensor");
  TciVerboseScope vs(ctx, "diag");
  vs.info = tci_shape_str(in);
  if (in->order == 1) {
    const int64_t n = in->shape[0];
    const int64_t shape[2] = {n, n};
    TCI_TRY(tci_zeros(ctx, in->dtype, 2, shape, out));
    if (n == 0) return TCI_OK;
    const int64_t st = in->strides[0];
    return dispatch(ctx, in->dtype, [&](auto tag) {
      using T = decltype(tag);
      k_diag_promote<T><<<grid_for(ctx, n), 256, 0, ctx->stream>>>((const T*)in->data, st, (T*)(*out)->data, n);
    });
  } else if (in->order == 2) {
    const int64_t m = in->shape[0] < in->shape[1] ? in->shape[0] : in->shape[1];
    TCI_TRY(tci_allocate(ctx, in->dtype, 1, &m, out));
    if (m == 0) return TCI_OK;
    const int64_t step = in->strides[0] + in->strides[1];
    return dispatch(ctx, in->dtype, [&](auto tag) {
      using T = decltype(tag);
      k_diag_extract<T><<<grid_for(ctx, m), 256, 0, ctx->stream>>>((const T*)in->data, step, (T*)(*out)->data, m);
    });
  }
  return tci_fail(ctx, TCI_ERR_SHAPE, "diag: input must be first- or second-order (order %d)", in->order);
}

extern "C" tci_status tci_diag(tci_context ctx, tci_tensor t) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "diag: invalid tensor");
  tci_tensor out = nullptr;
  TCI_TRY(tci_diag_to(ctx, t, &out));
  adopt(ctx, t, out);
  return TCI_OK;
}
