// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tci_b300.h"

#define TCI_MAX_ORDER 8

struct tci_context_s {
  int magic;
  int device;
  cudaStream_t stream;
  tci_precision precision;
  int verbose;
  int num_sms;
  int split_chunk_k;    // K depth per hi*hi accumulation unit of the split GEMM
  int split_xchunk_k;   // K depth per cross-product accumulation unit
  uint64_t wait_limit_ns = 0;   // bounded device waits of the tensor-core kernels (0: 2 s)
  // host-side allocation-failure injection (TCI_FAULT_ALLOC="n:k", read at context
  // creation): pooled allocation number n of this context (0-based) fails k times
  // in a row before the pool is asked, as if the device were out of memory
  int64_t fault_alloc_at = -1;
  int fault_alloc_times = 0;
  int64_t pool_allocs = 0;   // pooled allocations requested so far
  std::string last_error;
  // device scratch for reductions and kernel status words (owned)
  double* d_scalars;   // 64 doubles
  int* d_status;       // 16 ints: [0] = timeout flag of bounded waits
  double* h_scalars;   // pinned host mirror, 64 doubles
};

struct tci_tensor_s {
  int magic;
  tci_dtype dtype;
  int order;
  int64_t shape[TCI_MAX_ORDER];
  int64_t strides[TCI_MAX_ORDER];
  void* data;     // address of element 0
  void* alloc;    // owned allocation (NULL when borrowed or empty)
  int device;
};

constexpr int kCtxMagic = 0x7c1c0de;
constexpr int kTenMagic = 0x7e115e5;

// ---------------------------------------------------------------- errors
tci_status tci_fail(tci_context ctx, tci_status s, const char* fmt, ...);
tci_status tci_cuda_fail(tci_context ctx, cudaError_t e, const char* where);
bool tci_ctx_ok(tci_context ctx);
bool tci_ten_ok(tci_tensor t);

#define TCI_CHECK_CTX(ctx)                                                      \
  do {                                                                          \
    if (!tci_ctx_ok(ctx)) return tci_fail(nullptr, TCI_ERR_INVALID_CONTEXT, "invalid context"); \
  } while (0)

#define TCI_CUDA(ctx, call)                                                     \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess) return tci_cuda_fail(ctx, _e, #call);                \
  } while (0)

#define TCI_TRY(call)                                                           \
  do {                                                                          \
    tci_status _s = (call);                                                     \
    if (_s != TCI_OK) return _s;                                                \
  } while (0)

// ---------------------------------------------------------------- verbose
// TCI_VERBOSE (App. C.3): one line per call at level >= 1, with device time
// at level 2.  A scope object logs on destruction.
struct TciVerboseScope {
  tci_context ctx;
  const char* name;
  std::string info;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TciVerboseScope(tci_context c, const char* n);
  ~TciVerboseScope();
};

// ---------------------------------------------------------------- helpers
size_t tci_elem_bytes(tci_dtype d);
int64_t tci_numel(const tci_tensor_s* t);
bool tci_is_rowmajor(const tci_tensor_s* t);
void tci_rowmajor_strides(int order, const int64_t* shape, int64_t* strides);
std::string tci_shape_str(const tci_tensor_s* t);

tci_status tci_dev_alloc(tci_context ctx, size_t bytes, void** p);
void tci_dev_free(void* p);

// Owning holder of a tensor handle for host drivers (freed on scope exit).
struct TciOwned {
  tci_tensor t = nullptr;
  TciOwned() = default;
  TciOwned(const TciOwned&) = delete;
  TciOwned& operator=(const TciOwned&) = delete;
  TciOwned(TciOwned&& o) noexcept : t(o.t) { o.t = nullptr; }
  ~TciOwned() {
    if (t) tci_tensor_free(&t);
  }
  void reset(tci_tensor x) {
    if (t) tci_tensor_free(&t);
    t = x;
  }
  tci_tensor release() {
    tci_tensor x = t;
    t = nullptr;
    return x;
  }
};

// Strided permute-copy on the device (kernel K8): dst is row-major over
// `shape`; src element (i0..i{n-1}) at offset sum_k i_k * src_strides[k].
tci_status tci_launch_permute_copy(tci_context ctx, tci_dtype dt, int order, const int64_t* shape,
                                   const void* src, const int64_t* src_strides, void* dst);
// Same with an arbitrary destination stride vector (used to scatter results).
tci_status tci_launch_strided_copy(tci_context ctx, tci_dtype dt, int order, const int64_t* shape,
                                   const void* src, const int64_t* src_strides, void* dst,
                                   const int64_t* dst_strides);

// Materialise t row-major into new owned storage (in place on the handle).
tci_status tci_materialise(tci_context ctx, tci_tensor t);

// FP64 dot / norm helpers used by norm and Lanczos (deterministic order).
tci_status tci_launch_sumsq(tci_context ctx, tci_dtype dt, const void* x, int64_t n, double* d_out);
tci_status tci_launch_scale(tci_context ctx, tci_dtype dt, void* x, int64_t n, double re, double im);

// ---------------------------------------------------------------- GEMM
// C[m*ldcm + n*ldcn] = sum_k A[m*sam + k*sak] * B[n*sbn + k*sbk] (beta = 0),
// native arithmetic of dtype (FP64 FMA for F64), SIMT tiled kernel.
tci_status tci_gemm_native(tci_context ctx, tci_dtype dt, int64_t M, int64_t N, int64_t K,
                           const void* A, int64_t sam, int64_t sak, const void* B, int64_t sbn,
                           int64_t sbk, void* C, int64_t scm, int64_t scn);
// Batched form: nbatch independent products, operand x of batch t at x + t*sxb.
tci_status tci_gemm_native_batched(tci_context ctx, tci_dtype dt, int64_t nbatch, int64_t M, int64_t N, int64_t K,
                                   const void* A, int64_t sab, int64_t sam, int64_t sak, const void* B, int64_t sbb,
                                   int64_t sbn, int64_t sbk, void* C, int64_t scb, int64_t scm, int64_t scn);
// The same with a caller-owned split-K workspace (used when ws_bytes covers
// tci_gemm_native_workspace; then nothing is allocated, e.g. inside a graph capture).
tci_status tci_gemm_native_batched_ws(tci_context ctx, tci_dtype dt, int64_t nbatch, int64_t M, int64_t N, int64_t K,
                                      const void* A, int64_t sab, int64_t sam, int64_t sak, const void* B, int64_t sbb,
                                      int64_t sbn, int64_t sbk, void* C, int64_t scb, int64_t scm, int64_t scn, void* ws,
                                      size_t ws_bytes);
// Bytes of split-K partial products the native GEMM of this shape needs (0: no split).
size_t tci_gemm_native_workspace(tci_context ctx, tci_dtype dt, int64_t nbatch, int64_t M, int64_t N, int64_t K);

// Split-BF16 tensor-core GEMM (tcgen05).  Operands are given as three
// bfloat16 piece planes each: A pieces [3][M][Kp] and B pieces [3][N][Kp]
// (K-major rows, Kp % 8 == 0, plane stride = rows*Kp).  C element (m, n) at
// C[m*scm + n*scn]: FP64 (out_mode = 0), FP32 (out_mode = 1) or a normalised
// FP32 pair {hi, lo} per element (out_mode = 2, hi + lo = the result).  products = 6
// or 3.  chunk_k: K depth of one hi*hi accumulation unit (multiple of 32);
// xchunk_k: K depth of one cross-product accumulation unit.  raster: tile
// order (0 m-fastest, G > 0 groups of G m-blocks with n fastest inside).
tci_status tci_gemm_split_bf16(tci_context ctx, int64_t M, int64_t N, int64_t Kp,
                               const void* Apieces, const void* Bpieces, void* C, int out_mode,
                               int64_t scm, int64_t scn, int products, int chunk_k, int xchunk_k,
                               int raster);
// Same on row ranges of larger piece matrices: the A / B planes are
// a_plane_rows*Kp / b_plane_rows*Kp elements apart (Apieces, Bpieces point at
// the first row of the range in plane 0).
tci_status tci_gemm_split_bf16_sub(tci_context ctx, int64_t M, int64_t N, int64_t Kp, const void* Apieces,
                                   int64_t a_plane_rows, const void* Bpieces, int64_t b_plane_rows, void* C,
                                   int out_mode, int64_t scm, int64_t scn, int products, int chunk_k, int xchunk_k,
                                   int raster);

// The same on one problem with FP64 output C[m*N + n], also forming the dot
// products of the output with nv vectors V_i = V + i*ldv (same flat layout)
// and its sum of squares in the epilogue: part[i*part_stride + b] receives CTA
// b's partial sum (i = nv: <C, C>); *grid_out = the CTA count (<= part_stride).
tci_status tci_gemm_split_bf16_dots(tci_context ctx, int64_t M, int64_t N, int64_t Kp, const void* Ap, const void* Bp,
                                    double* C, int products, int chunk_k, int xchunk_k, int raster, const double* V,
                                    int64_t ldv, int nv, double* part, int part_stride, int* grid_out);

// Configuration of the split GEMM chosen by the autotuner (or defaults).
struct tci_gemm_cfg {
  int chunk_k = 256;
  int xchunk_k = 1024;
  int raster = 0;
  int bn = 128;   // tile width (grouped plans may use 64)
};
// Time candidate configurations with `run` (which must launch the plan's
// work with the given configuration on ctx->stream) and return the fastest
// whose chunk_k <= max_chunk_k.  `key` identifies the plan shape in the
// autotune cache (file named by TCI_AUTOTUNE_CACHE, when set); a cached entry
// is used without timing.  raster_candidates: whether tile order is tuned.
tci_status tci_autotune(tci_context ctx, const std::string& key, int max_chunk_k, bool raster_candidates,
                        tci_status (*run)(void* arg, const tci_gemm_cfg& cfg), void* arg, tci_gemm_cfg* best,
                        double* best_ms, bool bn_candidates = false);

// Grouped split-BF16 GEMM: all problems run in one persistent launch.
struct tci_split_problem {
  const void* Ap;   // bf16 pieces [3][M][Kp], 16-byte aligned
  const void* Bp;   // bf16 pieces [3][N][Kp], 16-byte aligned
  int64_t M, N, Kp;
  void* C;          // element (m, n) at C[m*scm + n*scn]
  int out_mode;
  int64_t scm, scn;
  int64_t a_plane_rows = 0, b_plane_rows = 0;   // piece-plane stride in rows (0: M, N)
  // out_mode 3 (gate epilogue of one TEBD bond: rows (a, t1), columns
  // (b, t2, re/im), M = 2 g_chi, N = 4 g_chi; C unused): the bond dimension and
  // the complex offsets of its gate and theta in the buffers the launch is given
  int64_t g_chi = 0, g_off = 0, th_off = 0;
};
struct tci_split_group;
// bn: tile width (128, or 64 for groups of narrow problems)
tci_status tci_split_group_create(tci_context ctx, int n, const tci_split_problem* probs, tci_split_group** out,
                                  int bn = 128);
void tci_split_group_destroy(tci_split_group* g);
// gate_ptrs: device array {gate base, theta base} (complex64), read by the
// kernel; required when the group has gate-epilogue problems.
tci_status tci_split_group_launch(tci_context ctx, const tci_split_group* g, int products, int chunk_k, int xchunk_k,
                                  int raster, const void* const* gate_ptrs = nullptr);

// Captured launch sequence of a plan.  The sequence is captured once on a
// private stream (capture is not possible on the legacy default stream) and
// replayed on the context stream; kernel nodes whose pointer arguments change
// per call are updated with cudaGraphExecKernelNodeSetParams.
struct tci_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<cudaGraphNode_t> nodes;   // kernel nodes in the order of `funcs`
};
// Capture `body` (which launches on ctx->stream) into g and locate the kernel
// nodes of the listed device functions.
tci_status tci_graph_capture(tci_context ctx, tci_graph* g, tci_status (*body)(void*), void* arg,
                             const std::vector<const void*>& funcs);
void tci_graph_destroy(tci_graph* g);

// K0: split a strided FP64/FP32 operand into three bfloat16 planes, packed
// K-major: out[p*plane + r*Kp + k] for r < rows, k < Kp (zero for k >= K),
// plane = plane_rows*Kp (plane_rows = 0: rows; a row range of a larger piece
// matrix passes its own out and the full row count).  Element (r, k) of the
// source is at src[r*sr + k*sk].
tci_status tci_launch_split3(tci_context ctx, tci_dtype dt, const void* src, int64_t rows,
                             int64_t K, int64_t sr, int64_t sk, void* out, int64_t Kp, int64_t plane_rows = 0);
