// Context, tensor handles, queries and TCI tensor-manipulation calls
// (App. C.1 type system; App. C.2 read-only queries, construction,
// reshape/transpose, norm/normalize/scale/linear_combine/close, version;
// App. C.3 TCI_VERBOSE).
#include <cuComplex.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <unordered_map>

#include "tci_internal.cuh"

static thread_local std::string g_last_error_noctx;

// ====================================================================== errors
tci_status tci_fail(tci_context ctx, tci_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx && ctx->magic == kCtxMagic)
    ctx->last_error = buf;
  else
    g_last_error_noctx = buf;
  if (ctx && ctx->magic == kCtxMagic && ctx->verbose > 0) fprintf(stderr, "[tci] error %d: %s\n", (int)s, buf);
  return s;
}

tci_status tci_cuda_fail(tci_context ctx, cudaError_t e, const char* where) {
  return tci_fail(ctx, e == cudaErrorMemoryAllocation ? TCI_ERR_ALLOC : TCI_ERR_CUDA, "%s: %s", where,
                  cudaGetErrorString(e));
}

bool tci_ctx_ok(tci_context ctx) { return ctx && ctx->magic == kCtxMagic; }
bool tci_ten_ok(tci_tensor t) { return t && t->magic == kTenMagic; }

extern "C" const char* tci_version(void) { return "1.0"; }

extern "C" const char* tci_status_string(tci_status s) {
  switch (s) {
    case TCI_OK: return "TCI_OK";
    case TCI_ERR_INVALID_ARG: return "TCI_ERR_INVALID_ARG";
    case TCI_ERR_SHAPE: return "TCI_ERR_SHAPE";
    case TCI_ERR_LABEL: return "TCI_ERR_LABEL";
    case TCI_ERR_DTYPE: return "TCI_ERR_DTYPE";
    case TCI_ERR_UNSUPPORTED: return "TCI_ERR_UNSUPPORTED";
    case TCI_ERR_ALLOC: return "TCI_ERR_ALLOC";
    case TCI_ERR_CUDA: return "TCI_ERR_CUDA";
    case TCI_ERR_TIMEOUT: return "TCI_ERR_TIMEOUT";
    case TCI_ERR_INVALID_CONTEXT: return "TCI_ERR_INVALID_CONTEXT";
  }
  return "TCI_ERR_UNKNOWN";
}

extern "C" const char* tci_last_error(tci_context ctx) {
  if (tci_ctx_ok(ctx)) return ctx->last_error.c_str();
  return g_last_error_noctx.c_str();
}

// ====================================================================== verbose
TciVerboseScope::TciVerboseScope(tci_context c, const char* n) : ctx(c), name(n) {
  if (tci_ctx_ok(ctx) && ctx->verbose >= 2) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, ctx->stream);
  }
}

TciVerboseScope::~TciVerboseScope() {
  if (!tci_ctx_ok(ctx) || ctx->verbose <= 0) return;
  if (ctx->verbose >= 2 && e0) {
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    fprintf(stderr, "[tci] %s %s time=%.3f ms\n", name, info.c_str(), ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  } else {
    fprintf(stderr, "[tci] %s %s\n", name, info.c_str());
  }
}

#define TCI_CHECK_TEN(ctx, t)                                                              \
  do {                                                                                     \
    TCI_CHECK_CTX(ctx);                                                                    \
    if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "invalid tensor handle"); \
  } while (0)

// ====================================================================== helpers
size_t tci_elem_bytes(tci_dtype d) {
  switch (d) {
    case TCI_F32: return 4;
    case TCI_F64: return 8;
    case TCI_C64: return 8;
    case TCI_C128: return 16;
  }
  return 0;
}

int64_t tci_numel(const tci_tensor_s* t) {
  int64_t n = 1;
  for (int i = 0; i < t->order; ++i) n *= t->shape[i];
  return n;
}

void tci_rowmajor_strides(int order, const int64_t* shape, int64_t* strides) {
  int64_t s = 1;
  for (int i = order - 1; i >= 0; --i) {
    strides[i] = s;
    s *= shape[i] > 0 ? shape[i] : 1;
  }
}

bool tci_is_rowmajor(const tci_tensor_s* t) {
  int64_t s = 1;
  for (int i = t->order - 1; i >= 0; --i) {
    if (t->shape[i] != 1 && t->strides[i] != s) return false;
    s *= t->shape[i];
  }
  return true;
}

std::string tci_shape_str(const tci_tensor_s* t) {
  static const char* names[] = {"f32", "f64", "c64", "c128"};
  std::string s = names[t->dtype];
  s += "{";
  for (int i = 0; i < t->order; ++i) {
    if (i) s += ",";
    s += std::to_string(t->shape[i]);
  }
  s += "}";
  return s;
}

// ---------------------------------------------------------------- device memory
// Library allocations are stream-ordered: they come from one memory pool per
// device (cudaMallocFromPoolAsync on the context's stream) and are returned
// with cudaFreeAsync on the stream they were allocated on, so the temporaries
// of a call never synchronise the device the way cudaMalloc / cudaFree do.
// The pool keeps up to kPoolKeepBytes of freed memory for reuse; more is
// returned to the CUDA driver at the next synchronisation.  Memory allocated while
// the context's stream is being captured into a graph, or without a context,
// comes from plain cudaMalloc.
namespace {

constexpr uint64_t kPoolKeepBytes = 8ull << 30;
constexpr int kMaxDevices = 64;

struct DevicePools {
  std::mutex mu;
  cudaMemPool_t pool[kMaxDevices] = {};
  std::unordered_map<void*, cudaStream_t> stream_of;   // live pool allocations
};

DevicePools& device_pools() {
  static DevicePools* p = new DevicePools();   // never destroyed: frees may run during exit
  return *p;
}

cudaMemPool_t pool_of(int device) {
  if (device < 0 || device >= kMaxDevices) return nullptr;
  DevicePools& dp = device_pools();
  std::lock_guard<std::mutex> lk(dp.mu);
  if (!dp.pool[device]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = kPoolKeepBytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    dp.pool[device] = pool;
  }
  return dp.pool[device];
}

}  // namespace

tci_status tci_dev_alloc(tci_context ctx, size_t bytes, void** p) {
  *p = nullptr;
  if (bytes == 0) return TCI_OK;
  cudaError_t e = cudaSuccess;
  if (tci_ctx_ok(ctx)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) {
      cudaGetLastError();
      cs = cudaStreamCaptureStatusActive;
    }
    cudaMemPool_t pool = cs == cudaStreamCaptureStatusNone ? pool_of(ctx->device) : nullptr;
    if (pool) {
      // injected failures (TCI_FAULT_ALLOC) stand in for the pool's answer on the host
      int injected = ctx->pool_allocs == ctx->fault_alloc_at ? ctx->fault_alloc_times : 0;
      ++ctx->pool_allocs;
      e = injected-- > 0 ? cudaErrorMemoryAllocation : cudaMallocFromPoolAsync(p, bytes, pool, ctx->stream);
      if (e == cudaErrorMemoryAllocation) {   // give cached memory back and try once more
        cudaGetLastError();
        cudaStreamSynchronize(ctx->stream);
        cudaMemPoolTrimTo(pool, 0);
        if (ctx->verbose > 0)
          fprintf(stderr, "[tci] pool: allocation of %zu bytes failed; pool trimmed, retrying once\n", bytes);
        e = injected-- > 0 ? cudaErrorMemoryAllocation : cudaMallocFromPoolAsync(p, bytes, pool, ctx->stream);
      }
      if (e == cudaSuccess) {
        DevicePools& dp = device_pools();
        std::lock_guard<std::mutex> lk(dp.mu);
        dp.stream_of[*p] = ctx->stream;
        return TCI_OK;
      }
      cudaGetLastError();
      *p = nullptr;
      return tci_fail(ctx, TCI_ERR_ALLOC, "device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
  }
  e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return tci_fail(ctx, TCI_ERR_ALLOC, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  return TCI_OK;
}

void tci_dev_free(void* p) {
  if (!p) return;
  cudaStream_t s = nullptr;
  bool pooled = false;
  {
    DevicePools& dp = device_pools();
    std::lock_guard<std::mutex> lk(dp.mu);
    auto it = dp.stream_of.find(p);
    if (it != dp.stream_of.end()) {
      s = it->second;
      pooled = true;
      dp.stream_of.erase(it);
    }
  }
  if (pooled)
    cudaFreeAsync(p, s);
  else
    cudaFree(p);
}

static bool valid_dtype(int d) { return d >= 0 && d <= 3; }

// ====================================================================== context
extern "C" tci_status tci_create_context(tci_context* out, int device, void* stream) {
  if (!out) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "create_context: NULL output");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return tci_cuda_fail(nullptr, e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev)
    return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "create_context: device %d out of range (%d devices)", device, ndev);
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return tci_cuda_fail(nullptr, e, "cudaSetDevice");
  tci_context ctx = new tci_context_s();
  ctx->magic = kCtxMagic;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  ctx->precision = TCI_PREC_NATIVE;
  ctx->split_chunk_k = 256;
  ctx->split_xchunk_k = 1024;
  const char* v = getenv("TCI_VERBOSE");
  ctx->verbose = v ? atoi(v) : 0;
  if (const char* f = getenv("TCI_FAULT_ALLOC")) {
    long long at = -1;
    int times = 0;
    if (sscanf(f, "%lld:%d", &at, &times) == 2 && at >= 0 && times > 0) {
      ctx->fault_alloc_at = at;
      ctx->fault_alloc_times = times;
    }
  }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  ctx->d_scalars = nullptr;
  ctx->d_status = nullptr;
  ctx->h_scalars = nullptr;
  if (cudaMalloc((void**)&ctx->d_scalars, 64 * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_status, 16 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_scalars, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    tci_dev_free(ctx->d_scalars);
    tci_dev_free(ctx->d_status);
    if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
    ctx->magic = 0;
    delete ctx;
    return tci_fail(nullptr, TCI_ERR_ALLOC, "create_context: scratch allocation failed");
  }
  cudaMemset(ctx->d_status, 0, 16 * sizeof(int));
  *out = ctx;
  if (ctx->verbose > 0) fprintf(stderr, "[tci] create_context device=%d stream=%p\n", device, stream);
  return TCI_OK;
}

extern "C" tci_status tci_destroy_context(tci_context* pctx) {
  if (!pctx || !tci_ctx_ok(*pctx)) return tci_fail(nullptr, TCI_ERR_INVALID_CONTEXT, "destroy_context: invalid context");
  tci_context ctx = *pctx;
  if (ctx->verbose > 0) fprintf(stderr, "[tci] destroy_context\n");
  cudaStreamSynchronize(ctx->stream);
  tci_dev_free(ctx->d_scalars);
  tci_dev_free(ctx->d_status);
  if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
  ctx->magic = 0;
  delete ctx;
  *pctx = nullptr;
  return TCI_OK;
}

extern "C" tci_status tci_context_set_stream(tci_context ctx, void* stream) {
  TCI_CHECK_CTX(ctx);
  ctx->stream = (cudaStream_t)stream;
  return TCI_OK;
}

extern "C" tci_status tci_context_set_precision(tci_context ctx, tci_precision p) {
  TCI_CHECK_CTX(ctx);
  if ((int)p < 0 || (int)p > 2) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "set_precision: unknown mode %d", (int)p);
  ctx->precision = p;
  return TCI_OK;
}

extern "C" tci_status tci_context_set_split_chunks(tci_context ctx, int chunk_k, int xchunk_k) {
  TCI_CHECK_CTX(ctx);
  if (chunk_k < 32 || chunk_k % 32 != 0 || xchunk_k < chunk_k || xchunk_k % chunk_k != 0)
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "set_split_chunks: need 32 | chunk_k and chunk_k | xchunk_k");
  ctx->split_chunk_k = chunk_k;
  ctx->split_xchunk_k = xchunk_k;
  return TCI_OK;
}

extern "C" tci_status tci_context_set_wait_limit(tci_context ctx, uint64_t limit_ns) {
  TCI_CHECK_CTX(ctx);
  ctx->wait_limit_ns = limit_ns;
  return TCI_OK;
}

extern "C" tci_status tci_context_get_precision(tci_context ctx, tci_precision* p) {
  TCI_CHECK_CTX(ctx);
  if (!p) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "get_precision: NULL output");
  *p = ctx->precision;
  return TCI_OK;
}

extern "C" tci_status tci_synchronize(tci_context ctx) {
  TCI_CHECK_CTX(ctx);
  TCI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int st = 0;
  TCI_CUDA(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    cudaMemset(ctx->d_status, 0, sizeof(int));
    return tci_fail(ctx, TCI_ERR_TIMEOUT, "a bounded device wait expired (status %d)", st);
  }
  return TCI_OK;
}

// ====================================================================== tensors
static tci_status new_tensor(tci_context ctx, tci_dtype dt, int order, const int64_t* shape,
                             const int64_t* strides, tci_tensor* out) {
  if (!out) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL tensor output");
  *out = nullptr;
  if (!valid_dtype(dt)) return tci_fail(ctx, TCI_ERR_DTYPE, "unknown dtype %d", (int)dt);
  if (order < 0 || order > TCI_MAX_ORDER) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "order %d outside 0..%d", order, TCI_MAX_ORDER);
  if (order > 0 && !shape) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL shape");
  tci_tensor t = new tci_tensor_s();
  t->magic = kTenMagic;
  t->dtype = dt;
  t->order = order;
  for (int i = 0; i < order; ++i) {
    if (shape[i] < 0) {
      delete t;
      return tci_fail(ctx, TCI_ERR_INVALID_ARG, "negative bond dimension");
    }
    t->shape[i] = shape[i];
  }
  if (strides) {
    for (int i = 0; i < order; ++i) {
      if (strides[i] < 0) {
        delete t;
        return tci_fail(ctx, TCI_ERR_INVALID_ARG, "negative stride");
      }
      t->strides[i] = strides[i];
    }
  } else {
    tci_rowmajor_strides(order, t->shape, t->strides);
  }
  t->data = nullptr;
  t->alloc = nullptr;
  t->device = ctx->device;
  *out = t;
  return TCI_OK;
}

extern "C" tci_status tci_tensor_wrap(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape,
                                      const int64_t* strides, void* data, tci_tensor* out) {
  TCI_CHECK_CTX(ctx);
  TCI_TRY(new_tensor(ctx, dtype, order, shape, strides, out));
  if (!data && tci_numel(*out) > 0) {
    delete *out;
    *out = nullptr;
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tensor_wrap: NULL data for a non-empty tensor");
  }
  (*out)->data = data;
  return TCI_OK;
}

static tci_status alloc_tensor(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape, tci_tensor* out,
                               bool zero) {
  TCI_CHECK_CTX(ctx);
  TCI_TRY(new_tensor(ctx, dtype, order, shape, nullptr, out));
  size_t bytes = (size_t)tci_numel(*out) * tci_elem_bytes(dtype);
  tci_status s = tci_dev_alloc(ctx, bytes, &(*out)->alloc);
  if (s != TCI_OK) {
    delete *out;
    *out = nullptr;
    return s;
  }
  (*out)->data = (*out)->alloc;
  if (zero && bytes) TCI_CUDA(ctx, cudaMemsetAsync((*out)->data, 0, bytes, ctx->stream));
  return TCI_OK;
}

extern "C" tci_status tci_allocate(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape, tci_tensor* out) {
  TciVerboseScope vs(ctx, "allocate");
  return alloc_tensor(ctx, dtype, order, shape, out, false);
}

extern "C" tci_status tci_zeros(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape, tci_tensor* out) {
  TciVerboseScope vs(ctx, "zeros");
  return alloc_tensor(ctx, dtype, order, shape, out, true);
}

extern "C" tci_status tci_tensor_free(tci_tensor* pt) {
  if (!pt || !tci_ten_ok(*pt)) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "tensor_free: invalid tensor");
  tci_tensor t = *pt;
  tci_dev_free(t->alloc);
  t->magic = 0;
  delete t;
  *pt = nullptr;
  return TCI_OK;
}

extern "C" tci_status tci_clear(tci_context ctx, tci_tensor t) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "clear: invalid tensor");
  TciVerboseScope vs(ctx, "clear");
  if (t->alloc) {
    cudaStreamSynchronize(ctx->stream);
    tci_dev_free(t->alloc);
  }
  t->alloc = nullptr;
  t->data = nullptr;
  t->order = 0;
  return TCI_OK;
}

extern "C" tci_status tci_move(tci_context ctx, tci_tensor from, tci_tensor* to) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(from) || !to) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "move: invalid tensor");
  TciVerboseScope vs(ctx, "move");
  tci_tensor t = new tci_tensor_s(*from);
  from->alloc = nullptr;
  from->data = nullptr;
  from->order = 0;
  *to = t;
  return TCI_OK;
}

extern "C" tci_status tci_copy(tci_context ctx, tci_tensor in, tci_tensor* out) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(in)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "copy: invalid tensor");
  TciVerboseScope vs(ctx, "copy");
  vs.info = tci_shape_str(in);
  TCI_TRY(alloc_tensor(ctx, in->dtype, in->order, in->shape, out, false));
  int64_t n = tci_numel(in);
  if (n == 0) return TCI_OK;
  if (tci_is_rowmajor(in)) {
    TCI_CUDA(ctx, cudaMemcpyAsync((*out)->data, in->data, n * tci_elem_bytes(in->dtype), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    return TCI_OK;
  }
  return tci_launch_permute_copy(ctx, in->dtype, in->order, in->shape, in->data, in->strides, (*out)->data);
}

// ---------------------------------------------------------------- queries

extern "C" tci_status tci_order(tci_context ctx, tci_tensor t, int* order) {
  TCI_CHECK_TEN(ctx, t);
  if (!order) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL output");
  *order = t->order;
  return TCI_OK;
}
extern "C" tci_status tci_shape(tci_context ctx, tci_tensor t, int64_t* shape) {
  TCI_CHECK_TEN(ctx, t);
  if (!shape && t->order) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL output");
  for (int i = 0; i < t->order; ++i) shape[i] = t->shape[i];
  return TCI_OK;
}
extern "C" tci_status tci_strides(tci_context ctx, tci_tensor t, int64_t* strides) {
  TCI_CHECK_TEN(ctx, t);
  if (!strides && t->order) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL output");
  for (int i = 0; i < t->order; ++i) strides[i] = t->strides[i];
  return TCI_OK;
}
extern "C" tci_status tci_size(tci_context ctx, tci_tensor t, int64_t* size) {
  TCI_CHECK_TEN(ctx, t);
  if (!size) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL output");
  *size = tci_numel(t);
  return TCI_OK;
}
extern "C" tci_status tci_size_bytes(tci_context ctx, tci_tensor t, int64_t* bytes) {
  TCI_CHECK_TEN(ctx, t);
  if (!bytes) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL output");
  *bytes = tci_numel(t) * (int64_t)tci_elem_bytes(t->dtype);
  return TCI_OK;
}
extern "C" tci_status tci_get_dtype(tci_context ctx, tci_tensor t, tci_dtype* dtype) {
  TCI_CHECK_TEN(ctx, t);
  if (!dtype) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL output");
  *dtype = t->dtype;
  return TCI_OK;
}
extern "C" tci_status tci_data(tci_context ctx, tci_tensor t, void** data) {
  TCI_CHECK_TEN(ctx, t);
  if (!data) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "NULL output");
  *data = t->data;
  return TCI_OK;
}

// ---------------------------------------------------------------- host transfer
extern "C" tci_status tci_to_host(tci_context ctx, tci_tensor t, void* host) {
  TCI_CHECK_TEN(ctx, t);
  TciVerboseScope vs(ctx, "to_host");
  const int64_t n = tci_numel(t);
  if (n == 0) return TCI_OK;
  if (!host) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "to_host: NULL host buffer");
  const size_t bytes = (size_t)n * tci_elem_bytes(t->dtype);
  tci_tensor tmp = nullptr;
  const void* src = t->data;
  if (!tci_is_rowmajor(t)) {
    TCI_TRY(tci_copy(ctx, t, &tmp));
    src = tmp->data;
  }
  cudaError_t e = cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (tmp) tci_tensor_free(&tmp);
  if (e != cudaSuccess) return tci_cuda_fail(ctx, e, "to_host");
  return TCI_OK;
}

extern "C" tci_status tci_from_host(tci_context ctx, tci_tensor t, const void* host) {
  TCI_CHECK_TEN(ctx, t);
  TciVerboseScope vs(ctx, "from_host");
  const int64_t n = tci_numel(t);
  if (n == 0) return TCI_OK;
  if (!host) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "from_host: NULL host buffer");
  const size_t bytes = (size_t)n * tci_elem_bytes(t->dtype);
  if (tci_is_rowmajor(t)) {
    TCI_CUDA(ctx, cudaMemcpyAsync(t->data, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    TCI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TCI_OK;
  }
  void* tmp = nullptr;
  TCI_TRY(tci_dev_alloc(ctx, bytes, &tmp));
  int64_t rm[TCI_MAX_ORDER];
  tci_rowmajor_strides(t->order, t->shape, rm);
  cudaError_t e = cudaMemcpyAsync(tmp, host, bytes, cudaMemcpyHostToDevice, ctx->stream);
  tci_status s = e == cudaSuccess ? tci_launch_strided_copy(ctx, t->dtype, t->order, t->shape, tmp, rm, t->data, t->strides)
                                  : tci_cuda_fail(ctx, e, "from_host");
  cudaStreamSynchronize(ctx->stream);
  tci_dev_free(tmp);
  return s;
}

// ---------------------------------------------------------------- K8 permute
struct PermArgs {
  int order;
  int64_t shape[TCI_MAX_ORDER];
  int64_t sstr[TCI_MAX_ORDER];
  int64_t dstr[TCI_MAX_ORDER];
};

// One thread per element, grid-stride.  Index decode runs on the logical
// row-major index of `shape`; the innermost logical dim maps to adjacent
// threads, so whichever operand is unit-stride there is coalesced.
template <typename T>
__global__ void k_strided_copy(PermArgs a, int64_t n, const T* __restrict__ src, T* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i, so = 0, dof = 0;
    for (int k = a.order - 1; k >= 0; --k) {
      int64_t c = r % a.shape[k];
      r /= a.shape[k];
      so += c * a.sstr[k];
      dof += c * a.dstr[k];
    }
    dst[dof] = src[so];
  }
}

struct alignas(16) c128_t { double re, im; };

tci_status tci_launch_strided_copy(tci_context ctx, tci_dtype dt, int order, const int64_t* shape, const void* src,
                                   const int64_t* src_strides, void* dst, const int64_t* dst_strides) {
  PermArgs a;
  a.order = order;
  int64_t n = 1;
  for (int i = 0; i < order; ++i) {
    a.shape[i] = shape[i];
    a.sstr[i] = src_strides[i];
    a.dstr[i] = dst_strides[i];
    n *= shape[i];
  }
  if (n == 0) return TCI_OK;
  int threads = 256;
  int64_t blocks = (n + threads - 1) / threads;
  int64_t cap = (int64_t)ctx->num_sms * 16;
  if (blocks > cap) blocks = cap;
  switch (tci_elem_bytes(dt)) {
    case 4: k_strided_copy<float><<<(int)blocks, threads, 0, ctx->stream>>>(a, n, (const float*)src, (float*)dst); break;
    case 8: k_strided_copy<double><<<(int)blocks, threads, 0, ctx->stream>>>(a, n, (const double*)src, (double*)dst); break;
    case 16: k_strided_copy<c128_t><<<(int)blocks, threads, 0, ctx->stream>>>(a, n, (const c128_t*)src, (c128_t*)dst); break;
    default: return tci_fail(ctx, TCI_ERR_DTYPE, "strided copy: bad dtype");
  }
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

tci_status tci_launch_permute_copy(tci_context ctx, tci_dtype dt, int order, const int64_t* shape, const void* src,
                                   const int64_t* src_strides, void* dst) {
  int64_t dstr[TCI_MAX_ORDER];
  tci_rowmajor_strides(order, shape, dstr);
  return tci_launch_strided_copy(ctx, dt, order, shape, src, src_strides, dst, dstr);
}

tci_status tci_materialise(tci_context ctx, tci_tensor t) {
  if (tci_is_rowmajor(t)) return TCI_OK;
  void* p = nullptr;
  size_t bytes = (size_t)tci_numel(t) * tci_elem_bytes(t->dtype);
  TCI_TRY(tci_dev_alloc(ctx, bytes, &p));
  tci_status s = tci_launch_permute_copy(ctx, t->dtype, t->order, t->shape, t->data, t->strides, p);
  if (s != TCI_OK) {
    tci_dev_free(p);
    return s;
  }
  if (t->alloc) {
    cudaStreamSynchronize(ctx->stream);
    tci_dev_free(t->alloc);
  }
  t->alloc = p;
  t->data = p;
  tci_rowmajor_strides(t->order, t->shape, t->strides);
  return TCI_OK;
}

// ---------------------------------------------------------------- reshape / transpose
// Try to express `new_shape` over the current strides without moving data
// (the standard "view" test: every new dim must lie inside one run of old
// dims that are contiguous with respect to each other).
static bool reshape_view_strides(const tci_tensor_s* t, int order, const int64_t* ns, int64_t* out_strides) {
  // drop size-1 dims of the old tensor
  int64_t os[TCI_MAX_ORDER], ost[TCI_MAX_ORDER];
  int on = 0;
  for (int i = 0; i < t->order; ++i)
    if (t->shape[i] != 1) {
      os[on] = t->shape[i];
      ost[on] = t->strides[i];
      ++on;
    }
  int oi = 0;
  int ni = 0;
  while (ni < order) {
    if (ns[ni] == 1) {
      out_strides[ni] = 1;
      ++ni;
      continue;
    }
    if (oi >= on) return false;
    // group old dims [oi, oj) and new dims [ni, nj) with equal products
    int64_t po = os[oi], pn = ns[ni];
    int oj = oi + 1, nj = ni + 1;
    while (po != pn) {
      if (po < pn) {
        if (oj >= on) return false;
        po *= os[oj++];
      } else {
        if (nj >= order) return false;
        pn *= ns[nj++];
      }
    }
    // old group must be contiguous among itself
    for (int k = oi; k < oj - 1; ++k)
      if (ost[k] != ost[k + 1] * os[k + 1]) return false;
    int64_t s = ost[oj - 1];
    for (int k = nj - 1; k >= ni; --k) {
      out_strides[k] = s;
      s *= ns[k];
    }
    oi = oj;
    ni = nj;
  }
  return oi == on;
}

static tci_status check_new_shape(tci_context ctx, tci_tensor t, int order, const int64_t* ns) {
  if (order < 0 || order > TCI_MAX_ORDER) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "reshape: order %d", order);
  if (order && !ns) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "reshape: NULL shape");
  int64_t n = 1;
  for (int i = 0; i < order; ++i) {
    if (ns[i] < 0) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "reshape: negative dim");
    n *= ns[i];
  }
  if (n != tci_numel(t)) return tci_fail(ctx, TCI_ERR_SHAPE, "reshape: element count %lld != %lld", (long long)n, (long long)tci_numel(t));
  return TCI_OK;
}

extern "C" tci_status tci_reshape(tci_context ctx, tci_tensor t, int order, const int64_t* ns) {
  TCI_CHECK_TEN(ctx, t);
  TciVerboseScope vs(ctx, "reshape");
  vs.info = tci_shape_str(t);
  TCI_TRY(check_new_shape(ctx, t, order, ns));
  int64_t st[TCI_MAX_ORDER];
  if (!reshape_view_strides(t, order, ns, st)) {
    TCI_TRY(tci_materialise(ctx, t));
    tci_rowmajor_strides(order, ns, st);
  }
  t->order = order;
  for (int i = 0; i < order; ++i) {
    t->shape[i] = ns[i];
    t->strides[i] = st[i];
  }
  return TCI_OK;
}

extern "C" tci_status tci_reshape_to(tci_context ctx, tci_tensor in, int order, const int64_t* ns, tci_tensor* out) {
  TCI_CHECK_TEN(ctx, in);
  if (!out) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "reshape_to: NULL output");
  TCI_TRY(check_new_shape(ctx, in, order, ns));
  int64_t st[TCI_MAX_ORDER];
  if (reshape_view_strides(in, order, ns, st)) {
    TCI_TRY(new_tensor(ctx, in->dtype, order, ns, st, out));
    (*out)->data = in->data;
    return TCI_OK;
  }
  TCI_TRY(tci_copy(ctx, in, out));
  (*out)->order = order;
  for (int i = 0; i < order; ++i) (*out)->shape[i] = ns[i];
  tci_rowmajor_strides(order, ns, (*out)->strides);
  return TCI_OK;
}

static tci_status check_perm(tci_context ctx, int order, const int* p) {
  if (order && !p) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "transpose: NULL new_order");
  int seen[TCI_MAX_ORDER] = {0};
  for (int i = 0; i < order; ++i) {
    if (p[i] < 0 || p[i] >= order || seen[p[i]]) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "transpose: new_order is not a permutation");
    seen[p[i]] = 1;
  }
  return TCI_OK;
}

extern "C" tci_status tci_transpose(tci_context ctx, tci_tensor t, const int* p) {
  TCI_CHECK_TEN(ctx, t);
  TciVerboseScope vs(ctx, "transpose");
  vs.info = tci_shape_str(t);
  TCI_TRY(check_perm(ctx, t->order, p));
  int64_t sh[TCI_MAX_ORDER], st[TCI_MAX_ORDER];
  for (int i = 0; i < t->order; ++i) {
    sh[i] = t->shape[p[i]];
    st[i] = t->strides[p[i]];
  }
  for (int i = 0; i < t->order; ++i) {
    t->shape[i] = sh[i];
    t->strides[i] = st[i];
  }
  return TCI_OK;
}

extern "C" tci_status tci_transpose_to(tci_context ctx, tci_tensor in, const int* p, tci_tensor* out) {
  TCI_CHECK_TEN(ctx, in);
  TciVerboseScope vs(ctx, "transpose_to");
  vs.info = tci_shape_str(in);
  TCI_TRY(check_perm(ctx, in->order, p));
  tci_tensor_s view = *in;
  for (int i = 0; i < in->order; ++i) {
    view.shape[i] = in->shape[p[i]];
    view.strides[i] = in->strides[p[i]];
  }
  view.alloc = nullptr;
  return tci_copy(ctx, &view, out);
}

// ---------------------------------------------------------------- norm / scale
// Deterministic two-level reduction: a fixed grid writes per-block partial
// sums of |x|^2 (each block reduces its grid-stride slice in a fixed order),
// then one block adds the partials in index order.
constexpr int kRedBlocks = 1184;   // 8 x 148 SMs
constexpr int kRedThreads = 256;

template <typename T>
__device__ __forceinline__ double abs2(const T& v);
template <> __device__ __forceinline__ double abs2<float>(const float& v) { return (double)v * (double)v; }
template <> __device__ __forceinline__ double abs2<double>(const double& v) { return v * v; }
template <> __device__ __forceinline__ double abs2<float2>(const float2& v) { return (double)v.x * v.x + (double)v.y * v.y; }
template <> __device__ __forceinline__ double abs2<double2>(const double2& v) { return v.x * v.x + v.y * v.y; }

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void k_sumsq_partial(const T* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += abs2<T>(x[i]);
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = s;
}

tci_status tci_launch_sumsq(tci_context ctx, tci_dtype dt, const void* x, int64_t n, double* d_out) {
  static_assert(kRedBlocks <= 4096, "partials");
  double* part = nullptr;
  TCI_TRY(tci_dev_alloc(ctx, kRedBlocks * sizeof(double), (void**)&part));
  switch (dt) {
    case TCI_F32: k_sumsq_partial<float><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>((const float*)x, n, part); break;
    case TCI_F64: k_sumsq_partial<double><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>((const double*)x, n, part); break;
    case TCI_C64: k_sumsq_partial<float2><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>((const float2*)x, n, part); break;
    case TCI_C128: k_sumsq_partial<double2><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>((const double2*)x, n, part); break;
  }
  k_sum_partials<<<1, 1024, 0, ctx->stream>>>(part, kRedBlocks, d_out);
  cudaError_t e = cudaGetLastError();
  tci_dev_free(part);   // stream-ordered, after the two kernels
  if (e != cudaSuccess) return tci_cuda_fail(ctx, e, "sumsq kernels");
  return TCI_OK;
}

template <typename T, typename S>
__global__ void k_scale_real(T* x, int64_t n, S s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = x[i] * s;
}

template <typename C, typename S>
__global__ void k_scale_cplx(C* x, int64_t n, S re, S im) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    C v = x[i];
    C r;
    r.x = v.x * re - v.y * im;
    r.y = v.x * im + v.y * re;
    x[i] = r;
  }
}

tci_status tci_launch_scale(tci_context ctx, tci_dtype dt, void* x, int64_t n, double re, double im) {
  if (n == 0) return TCI_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
  switch (dt) {
    case TCI_F32: k_scale_real<float, float><<<(int)blocks, 256, 0, ctx->stream>>>((float*)x, n, (float)re); break;
    case TCI_F64: k_scale_real<double, double><<<(int)blocks, 256, 0, ctx->stream>>>((double*)x, n, re); break;
    case TCI_C64: k_scale_cplx<float2, float><<<(int)blocks, 256, 0, ctx->stream>>>((float2*)x, n, (float)re, (float)im); break;
    case TCI_C128: k_scale_cplx<double2, double><<<(int)blocks, 256, 0, ctx->stream>>>((double2*)x, n, re, im); break;
  }
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

// Element-wise kernels below operate on the logical elements; a strided
// tensor is materialised first (its handle then owns row-major storage).
static tci_status dense_view(tci_context ctx, tci_tensor t) {
  if (tci_is_rowmajor(t)) return TCI_OK;
  return tci_materialise(ctx, t);
}

extern "C" tci_status tci_norm(tci_context ctx, tci_tensor t, double* out) {
  TCI_CHECK_TEN(ctx, t);
  if (!out) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "norm: NULL output");
  TciVerboseScope vs(ctx, "norm");
  vs.info = tci_shape_str(t);
  int64_t n = tci_numel(t);
  if (n == 0) {
    *out = 0.0;
    return TCI_OK;
  }
  const void* data = t->data;
  tci_tensor tmp = nullptr;
  if (!tci_is_rowmajor(t)) {
    TCI_TRY(tci_copy(ctx, t, &tmp));
    data = tmp->data;
  }
  tci_status s = tci_launch_sumsq(ctx, t->dtype, data, n, ctx->d_scalars);
  if (s == TCI_OK) {
    cudaError_t e = cudaMemcpyAsync(ctx->h_scalars, ctx->d_scalars, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) s = tci_cuda_fail(ctx, e, "norm readback");
  }
  if (tmp) tci_tensor_free(&tmp);
  if (s != TCI_OK) return s;
  *out = sqrt(ctx->h_scalars[0]);
  return TCI_OK;
}

extern "C" tci_status tci_scale(tci_context ctx, tci_tensor t, double re, double im) {
  TCI_CHECK_TEN(ctx, t);
  TciVerboseScope vs(ctx, "scale");
  vs.info = tci_shape_str(t);
  TCI_TRY(dense_view(ctx, t));
  return tci_launch_scale(ctx, t->dtype, t->data, tci_numel(t), re, im);
}

extern "C" tci_status tci_normalize(tci_context ctx, tci_tensor t, double* old_norm) {
  TCI_CHECK_TEN(ctx, t);
  TciVerboseScope vs(ctx, "normalize");
  double nrm = 0.0;
  TCI_TRY(tci_norm(ctx, t, &nrm));
  if (old_norm) *old_norm = nrm;
  if (nrm == 0.0) return TCI_OK;
  return tci_scale(ctx, t, 1.0 / nrm, 0.0);
}

// ---------------------------------------------------------------- linear_combine
template <typename T, typename S>
__global__ void k_axpy_real(T* __restrict__ y, const T* __restrict__ x, int64_t n, S a, int first) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = first ? (T)(a * x[i]) : (T)(y[i] + a * x[i]);
}

extern "C" tci_status tci_linear_combine(tci_context ctx, int n, const tci_tensor* ins, const double* coefs,
                                         tci_tensor* out) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "linear_combine");
  if (n <= 0 || !ins || !out) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "linear_combine: empty input list");
  for (int i = 0; i < n; ++i) {
    if (!tci_ten_ok(ins[i])) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "linear_combine: invalid tensor %d", i);
    if (ins[i]->dtype != ins[0]->dtype) return tci_fail(ctx, TCI_ERR_DTYPE, "linear_combine: dtypes differ");
    if (ins[i]->order != ins[0]->order) return tci_fail(ctx, TCI_ERR_SHAPE, "linear_combine: shapes differ");
    for (int k = 0; k < ins[0]->order; ++k)
      if (ins[i]->shape[k] != ins[0]->shape[k]) return tci_fail(ctx, TCI_ERR_SHAPE, "linear_combine: shapes differ");
  }
  tci_tensor_s* t0 = ins[0];
  tci_tensor res = nullptr;
  TCI_TRY(alloc_tensor(ctx, t0->dtype, t0->order, t0->shape, &res, false));
  int64_t m = tci_numel(t0);
  int64_t blocks = (m + 255) / 256;
  if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
  if (blocks < 1) blocks = 1;
  bool is_real = t0->dtype == TCI_F32 || t0->dtype == TCI_F64;
  int64_t mm = is_real ? m : 2 * m;   // complex: scale re and im by the same real coefficient
  for (int i = 0; i < n; ++i) {
    const void* x = ins[i]->data;
    tci_tensor tmp = nullptr;
    if (!tci_is_rowmajor(ins[i])) {
      tci_status s = tci_copy(ctx, ins[i], &tmp);
      if (s != TCI_OK) {
        tci_tensor_free(&res);
        return s;
      }
      x = tmp->data;
    }
    double a = coefs ? coefs[i] : 1.0;
    if (t0->dtype == TCI_F32 || t0->dtype == TCI_C64)
      k_axpy_real<float, float><<<(int)blocks, 256, 0, ctx->stream>>>((float*)res->data, (const float*)x, mm, (float)a, i == 0);
    else
      k_axpy_real<double, double><<<(int)blocks, 256, 0, ctx->stream>>>((double*)res->data, (const double*)x, mm, a, i == 0);
    if (tmp) {
      cudaStreamSynchronize(ctx->stream);
      tci_tensor_free(&tmp);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    tci_tensor_free(&res);
    return tci_cuda_fail(ctx, e, "linear_combine kernels");
  }
  if (*out) {
    tci_tensor o = *out;
    if (!tci_ten_ok(o)) {
      tci_tensor_free(&res);
      return tci_fail(ctx, TCI_ERR_INVALID_ARG, "linear_combine: invalid output");
    }
    if (o->alloc || o->data == nullptr) {
      cudaStreamSynchronize(ctx->stream);
      tci_dev_free(o->alloc);
      o->alloc = res->alloc;
      o->data = res->data;
      o->dtype = res->dtype;
      o->order = res->order;
      for (int k = 0; k < res->order; ++k) {
        o->shape[k] = res->shape[k];
        o->strides[k] = res->strides[k];
      }
      res->alloc = nullptr;
      tci_tensor_free(&res);
      return TCI_OK;
    }
    // borrowed output: write the result into it
    bool same = o->dtype == res->dtype && o->order == res->order;
    for (int k = 0; same && k < res->order; ++k) same = o->shape[k] == res->shape[k];
    if (!same) {
      tci_tensor_free(&res);
      return tci_fail(ctx, TCI_ERR_SHAPE, "linear_combine: borrowed output has the wrong shape/dtype");
    }
    tci_status s = tci_launch_strided_copy(ctx, res->dtype, res->order, res->shape, res->data, res->strides, o->data,
                                           o->strides);
    cudaStreamSynchronize(ctx->stream);
    tci_tensor_free(&res);
    return s;
  }
  *out = res;
  return TCI_OK;
}

// ---------------------------------------------------------------- close
template <typename T>
__device__ __forceinline__ double absdiff(const T& a, const T& b);
template <> __device__ __forceinline__ double absdiff<float>(const float& a, const float& b) { return fabs((double)a - (double)b); }
template <> __device__ __forceinline__ double absdiff<double>(const double& a, const double& b) { return fabs(a - b); }
template <> __device__ __forceinline__ double absdiff<float2>(const float2& a, const float2& b) {
  return hypot((double)a.x - b.x, (double)a.y - b.y);
}
template <> __device__ __forceinline__ double absdiff<double2>(const double2& a, const double2& b) {
  return hypot(a.x - b.x, a.y - b.y);
}

template <typename T>
__global__ void k_maxdiff(const T* __restrict__ a, const T* __restrict__ b, int64_t n, unsigned long long* out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = absdiff<T>(a[i], b[i]);
    if (!(d <= m)) m = d;   // NaN propagates as +inf below
  }
  if (m != m) m = __longlong_as_double(0x7ff0000000000000ULL);
  // non-negative doubles order like their bit patterns
  for (int o = 16; o > 0; o >>= 1) {
    double other = __shfl_down_sync(0xffffffffu, m, o);
    m = other > m ? other : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

extern "C" tci_status tci_close(tci_context ctx, tci_tensor a, tci_tensor b, double eps, int* result) {
  TCI_CHECK_CTX(ctx);
  if (!tci_ten_ok(a) || !tci_ten_ok(b) || !result) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "close: invalid argument");
  if (eps < 0) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "close: epsilon must be >= 0");
  TciVerboseScope vs(ctx, "close");
  *result = 0;
  if (a->dtype != b->dtype) return tci_fail(ctx, TCI_ERR_DTYPE, "close: dtypes differ");
  if (a->order != b->order) return TCI_OK;
  for (int k = 0; k < a->order; ++k)
    if (a->shape[k] != b->shape[k]) return TCI_OK;
  int64_t n = tci_numel(a);
  if (n == 0) {
    *result = 1;
    return TCI_OK;
  }
  tci_tensor ta = nullptr, tb = nullptr;
  const void* pa = a->data;
  const void* pb = b->data;
  if (!tci_is_rowmajor(a)) {
    TCI_TRY(tci_copy(ctx, a, &ta));
    pa = ta->data;
  }
  if (!tci_is_rowmajor(b)) {
    tci_status s = tci_copy(ctx, b, &tb);
    if (s != TCI_OK) {
      if (ta) tci_tensor_free(&ta);
      return s;
    }
    pb = tb->data;
  }
  unsigned long long* dmax = (unsigned long long*)ctx->d_scalars;
  cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), ctx->stream);
  int blocks = (int)((n + 255) / 256);
  if (blocks > ctx->num_sms * 8) blocks = ctx->num_sms * 8;
  switch (a->dtype) {
    case TCI_F32: k_maxdiff<float><<<blocks, 256, 0, ctx->stream>>>((const float*)pa, (const float*)pb, n, dmax); break;
    case TCI_F64: k_maxdiff<double><<<blocks, 256, 0, ctx->stream>>>((const double*)pa, (const double*)pb, n, dmax); break;
    case TCI_C64: k_maxdiff<float2><<<blocks, 256, 0, ctx->stream>>>((const float2*)pa, (const float2*)pb, n, dmax); break;
    case TCI_C128: k_maxdiff<double2><<<blocks, 256, 0, ctx->stream>>>((const double2*)pa, (const double2*)pb, n, dmax); break;
  }
  cudaError_t e = cudaMemcpyAsync(ctx->h_scalars, dmax, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (ta) tci_tensor_free(&ta);
  if (tb) tci_tensor_free(&tb);
  if (e != cudaSuccess) return tci_cuda_fail(ctx, e, "close");
  *result = ctx->h_scalars[0] <= eps ? 1 : 0;
  return TCI_OK;
}

// ====================================================================== graphs
tci_status tci_graph_capture(tci_context ctx, tci_graph* g, tci_status (*body)(void*), void* arg,
                             const std::vector<const void*>& funcs) {
  if (!g->cap) TCI_CUDA(ctx, cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
  cudaStream_t saved = ctx->stream;
  TCI_CUDA(ctx, cudaStreamSynchronize(saved));
  ctx->stream = g->cap;
  cudaError_t e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
  tci_status s = e == cudaSuccess ? body(arg) : tci_cuda_fail(ctx, e, "cudaStreamBeginCapture");
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(g->cap, &graph);
  ctx->stream = saved;
  if (s != TCI_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e2 != cudaSuccess) return tci_cuda_fail(ctx, e2, "cudaStreamEndCapture");
  size_t n = 0;
  TCI_CUDA(ctx, cudaGraphGetNodes(graph, nullptr, &n));
  std::vector<cudaGraphNode_t> all(n);
  TCI_CUDA(ctx, cudaGraphGetNodes(graph, all.data(), &n));
  g->nodes.assign(funcs.size(), nullptr);
  for (cudaGraphNode_t nd : all) {
    cudaGraphNodeType ty;
    TCI_CUDA(ctx, cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    TCI_CUDA(ctx, cudaGraphKernelNodeGetParams(nd, &kp));
    for (size_t i = 0; i < funcs.size(); ++i)
      if (kp.func == funcs[i] && !g->nodes[i]) g->nodes[i] = nd;
  }
  for (auto nd : g->nodes)
    if (!nd) {
      cudaGraphDestroy(graph);
      return tci_fail(ctx, TCI_ERR_CUDA, "graph capture: kernel node not found");
    }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return tci_cuda_fail(ctx, e, "cudaGraphInstantiate");
  }
  g->graph = graph;
  g->exec = exec;
  return TCI_OK;
}

void tci_graph_destroy(tci_graph* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cap) cudaStreamDestroy(g->cap);
  g->exec = nullptr;
  g->graph = nullptr;
  g->cap = nullptr;
  g->nodes.clear();
}
