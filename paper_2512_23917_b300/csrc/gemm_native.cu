// Native-arithmetic strided GEMM (SIMT): C(m,n) = sum_k A(m,k) B(n,k),
// optionally batched (blockIdx.z; each operand advances by its batch stride).
// Operands are read in place through arbitrary (m,k)/(n,k) strides, so a
// permuted operand needs no materialised transpose.  FP64 on B300 has no
// fast tensor-core path, so a register-tiled FMA kernel is the FP64 roof.
// When the output has too few tiles to fill the SMs and K is long enough (a
// batch of small Gram-like products, or a small H_eff), K is split: each
// split writes a partial product and a second kernel adds the partials in
// split order.
#include <algorithm>

#include "tci_internal.cuh"

namespace {

template <typename T> struct Acc { using type = T; };

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 fma_(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 fma_(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ float add_(float a, float b) { return a + b; }
__device__ __forceinline__ double add_(double a, double b) { return a + b; }
__device__ __forceinline__ float2 add_(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 add_(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T zero_();
template <> __device__ __forceinline__ float zero_<float>() { return 0.f; }
template <> __device__ __forceinline__ double zero_<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 zero_<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_<double2>() { return make_double2(0.0, 0.0); }

// Tiles of BM x BN outputs, BK deep, TM x TN outputs per thread, 256 threads:
// 64 x 64 by default, 32 x 32 when 64-wide tiles cannot occupy every SM (an
// SM issues only 2 FP64 FMAs per clock, so small products must spread out).
constexpr int BK = 16;
constexpr int NT = 256;

// ACONT: 0 = operand contiguous (or best) along k, 1 = along m/n.
template <typename T, int ACONT, int BCONT, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(NT) k_gemm_strided(int64_t M, int64_t N, int64_t K, const T* __restrict__ A,
                                                     int64_t sam, int64_t sak, const T* __restrict__ B, int64_t sbn,
                                                     int64_t sbk, T* __restrict__ C, int64_t scm, int64_t scn,
                                                     int64_t sab, int64_t sbb, int64_t scb, int nsplit,
                                                     int64_t kchunk, int64_t scs) {
  __shared__ T As[BK][BM + 1];
  const int64_t bz = blockIdx.z / nsplit, split = blockIdx.z % nsplit;
  A += bz * sab;
  B += bz * sbb;
  C += bz * scb + split * scs;
  const int64_t kb = split * kchunk, ke = kb + kchunk < K ? kb + kchunk : K;
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = zero_<T>();

  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int e = tid + r * NT;
      int kk, mm;
      if (ACONT == 0) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < ke) ? A[gm * sam + gk * sak] : zero_<T>();
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      int e = tid + r * NT;
      int kk, nn;
      if (BCONT == 0) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      int64_t gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < ke) ? B[gn * sbn + gk * sbk] : zero_<T>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma_(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t gm = m0 + ty + i * (BM / TM);
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t gn = n0 + tx + j * (BN / TN);
      if (gn < N) C[gm * scm + gn * scn] = acc[i][j];
    }
  }
}

// C[b, m, n] = sum_s part[s][b][m][n] (splits added in order)
template <typename T>
__global__ void k_split_sum(const T* __restrict__ part, int nsplit, int64_t nb, int64_t M, int64_t N,
                            T* __restrict__ C, int64_t scb, int64_t scm, int64_t scn) {
  const int64_t per = nb * M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per; i += (int64_t)gridDim.x * blockDim.x) {
    T acc = part[i];
    for (int s = 1; s < nsplit; ++s) acc = add_(acc, part[s * per + i]);
    const int64_t b = i / (M * N), r = i - b * (M * N), m = r / N, n = r - m * N;
    C[b * scb + m * scm + n * scn] = acc;
  }
}

// K split of a launch: split count and depth per split (nsplit = 1: no split).
void split_of(tci_context ctx, int64_t nbatch, int64_t M, int64_t N, int64_t K, int BM, int BN, int64_t* nsplit_out,
              int64_t* kchunk_out) {
  const int64_t tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM) * nbatch, want = 2 * (int64_t)ctx->num_sms;
  // split K when the tiles cannot fill two waves and each split keeps >= 32 of K
  int64_t nsplit = 1;
  if (tiles < want && K >= 64) {
    nsplit = std::min<int64_t>({(want + tiles - 1) / tiles, K / 32, 16});
    if (nsplit < 1) nsplit = 1;
  }
  int64_t kchunk = K;
  if (nsplit > 1) {
    kchunk = ((K + nsplit - 1) / nsplit + BK - 1) / BK * BK;
    nsplit = (K + kchunk - 1) / kchunk;
  }
  *nsplit_out = nsplit;
  *kchunk_out = kchunk;
}

// 64 x 64 tiles unless they cannot occupy every SM
bool small_tiles(tci_context ctx, int64_t nbatch, int64_t M, int64_t N) {
  return ((M + 63) / 64) * ((N + 63) / 64) * nbatch < (int64_t)ctx->num_sms;
}

template <typename T, int BM, int BN, int TM, int TN>
tci_status launch_tiles(tci_context ctx, int64_t nbatch, int64_t M, int64_t N, int64_t K, const void* A, int64_t sab,
                        int64_t sam, int64_t sak, const void* B, int64_t sbb, int64_t sbn, int64_t sbk, void* C,
                        int64_t scb, int64_t scm, int64_t scn, void* ws, size_t ws_bytes) {
  static_assert((BM / TM) * (BN / TN) == NT, "tile shape");
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  if (grid.y > 65535u) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "gemm: M too large for the native kernel");
  int ac = (sak == 1 || sam != 1) ? 0 : 1;
  int bc = (sbk == 1 || sbn != 1) ? 0 : 1;
  int64_t nsplit, kchunk;
  split_of(ctx, nbatch, M, N, K, BM, BN, &nsplit, &kchunk);
  T* part = nullptr;
  const int64_t per = nbatch * M * N;
  const bool own = nsplit > 1 && !(ws && ws_bytes >= sizeof(T) * nsplit * per);   // else the caller's workspace
  if (nsplit > 1) {
    if (own) TCI_TRY(tci_dev_alloc(ctx, sizeof(T) * nsplit * per, (void**)&part));
    else part = (T*)ws;
  }
  T* cout = nsplit > 1 ? part : (T*)C;
  const int64_t ocb = nsplit > 1 ? M * N : scb, ocm = nsplit > 1 ? N : scm, ocn = nsplit > 1 ? 1 : scn;
  const int64_t bmax = 65535 / nsplit;
  tci_status st = TCI_OK;
  for (int64_t b0 = 0; b0 < nbatch && st == TCI_OK; b0 += bmax) {
    const int64_t nb = nbatch - b0 < bmax ? nbatch - b0 : bmax;
    grid.z = (unsigned)(nb * nsplit);
    const T* a = (const T*)A + b0 * sab;
    const T* b = (const T*)B + b0 * sbb;
    T* c = cout + b0 * ocb;
    const int ns = (int)nsplit;
    if (ac == 0 && bc == 0)
      k_gemm_strided<T, 0, 0, BM, BN, TM, TN><<<grid, NT, 0, ctx->stream>>>(M, N, K, a, sam, sak, b, sbn, sbk, c, ocm,
                                                                            ocn, sab, sbb, ocb, ns, kchunk, per);
    else if (ac == 0 && bc == 1)
      k_gemm_strided<T, 0, 1, BM, BN, TM, TN><<<grid, NT, 0, ctx->stream>>>(M, N, K, a, sam, sak, b, sbn, sbk, c, ocm,
                                                                            ocn, sab, sbb, ocb, ns, kchunk, per);
    else if (ac == 1 && bc == 0)
      k_gemm_strided<T, 1, 0, BM, BN, TM, TN><<<grid, NT, 0, ctx->stream>>>(M, N, K, a, sam, sak, b, sbn, sbk, c, ocm,
                                                                            ocn, sab, sbb, ocb, ns, kchunk, per);
    else
      k_gemm_strided<T, 1, 1, BM, BN, TM, TN><<<grid, NT, 0, ctx->stream>>>(M, N, K, a, sam, sak, b, sbn, sbk, c, ocm,
                                                                            ocn, sab, sbb, ocb, ns, kchunk, per);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = tci_cuda_fail(ctx, e, "gemm launch");
  }
  if (nsplit > 1) {
    if (st == TCI_OK) {
      const int64_t blocks = std::min<int64_t>((per + 255) / 256, (int64_t)ctx->num_sms * 16);
      k_split_sum<T><<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, ctx->stream>>>(part, (int)nsplit, nbatch, M, N,
                                                                                       (T*)C, scb, scm, scn);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = tci_cuda_fail(ctx, e, "gemm split sum");
    }
    if (own) tci_dev_free(part);
  }
  return st;
}

template <typename T>
tci_status launch(tci_context ctx, int64_t nbatch, int64_t M, int64_t N, int64_t K, const void* A, int64_t sab,
                  int64_t sam, int64_t sak, const void* B, int64_t sbb, int64_t sbn, int64_t sbk, void* C, int64_t scb,
                  int64_t scm, int64_t scn, void* ws, size_t ws_bytes) {
  if (small_tiles(ctx, nbatch, M, N))
    return launch_tiles<T, 32, 32, 2, 2>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn,
                                         ws, ws_bytes);
  return launch_tiles<T, 64, 64, 4, 4>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn, ws,
                                       ws_bytes);
}

}  // namespace

tci_status tci_gemm_native_batched_ws(tci_context ctx, tci_dtype dt, int64_t nbatch, int64_t M, int64_t N, int64_t K,
                                      const void* A, int64_t sab, int64_t sam, int64_t sak, const void* B, int64_t sbb,
                                      int64_t sbn, int64_t sbk, void* C, int64_t scb, int64_t scm, int64_t scn, void* ws,
                                      size_t ws_bytes) {
  if (nbatch <= 0 || M == 0 || N == 0) return TCI_OK;
  switch (dt) {
    case TCI_F32:
      return launch<float>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn, ws, ws_bytes);
    case TCI_F64:
      return launch<double>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn, ws, ws_bytes);
    case TCI_C64:
      return launch<float2>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn, ws, ws_bytes);
    case TCI_C128:
      return launch<double2>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn, ws, ws_bytes);
  }
  return tci_fail(ctx, TCI_ERR_DTYPE, "gemm: bad dtype");
}

size_t tci_gemm_native_workspace(tci_context ctx, tci_dtype dt, int64_t nbatch, int64_t M, int64_t N, int64_t K) {
  if (nbatch <= 0 || M == 0 || N == 0) return 0;
  const bool st = small_tiles(ctx, nbatch, M, N);
  int64_t nsplit, kchunk;
  split_of(ctx, nbatch, M, N, K, st ? 32 : 64, st ? 32 : 64, &nsplit, &kchunk);
  return nsplit > 1 ? tci_elem_bytes(dt) * (size_t)(nsplit * nbatch * M * N) : 0;
}

tci_status tci_gemm_native_batched(tci_context ctx, tci_dtype dt, int64_t nbatch, int64_t M, int64_t N, int64_t K,
                                   const void* A, int64_t sab, int64_t sam, int64_t sak, const void* B, int64_t sbb,
                                   int64_t sbn, int64_t sbk, void* C, int64_t scb, int64_t scm, int64_t scn) {
  return tci_gemm_native_batched_ws(ctx, dt, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn,
                                    nullptr, 0);
}

tci_status tci_gemm_native(tci_context ctx, tci_dtype dt, int64_t M, int64_t N, int64_t K, const void* A, int64_t sam,
                           int64_t sak, const void* B, int64_t sbn, int64_t sbk, void* C, int64_t scm, int64_t scn) {
  return tci_gemm_native_batched(ctx, dt, 1, M, N, K, A, 0, sam, sak, B, 0, sbn, sbk, C, 0, scm, scn);
}
