// Native-arithmetic strided GEMM (SIMT): C(m,n) = sum_k A(m,k) B(n,k),
// optionally batched (blockIdx.z; each operand advances by its batch stride).
// Operands are read in place through arbitrary (m,k)/(n,k) strides, so a
// permuted operand needs no materialised transpose.  FP64 on B300 has no
// fast tensor-core path, so a register-tiled FMA kernel is the FP64 roof.
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
template <typename T> __device__ __forceinline__ T zero_();
template <> __device__ __forceinline__ float zero_<float>() { return 0.f; }
template <> __device__ __forceinline__ double zero_<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 zero_<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_<double2>() { return make_double2(0.0, 0.0); }

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
constexpr int NT = (BM / TM) * (BN / TN);   // 256 threads

// ACONT: 0 = operand contiguous (or best) along k, 1 = along m/n.
template <typename T, int ACONT, int BCONT>
__global__ void __launch_bounds__(NT) k_gemm_strided(int64_t M, int64_t N, int64_t K, const T* __restrict__ A,
                                                     int64_t sam, int64_t sak, const T* __restrict__ B, int64_t sbn,
                                                     int64_t sbk, T* __restrict__ C, int64_t scm, int64_t scn,
                                                     int64_t sab, int64_t sbb, int64_t scb) {
  __shared__ T As[BK][BM + 1];
  A += (int64_t)blockIdx.z * sab;
  B += (int64_t)blockIdx.z * sbb;
  C += (int64_t)blockIdx.z * scb;
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = zero_<T>();

  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int e = tid + r * NT;
      int kk, mm;
      if (ACONT == 0) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : zero_<T>();
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      int e = tid + r * NT;
      int kk, nn;
      if (BCONT == 0) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      int64_t gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? B[gn * sbn + gk * sbk] : zero_<T>();
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

template <typename T>
tci_status launch(tci_context ctx, int64_t nbatch, int64_t M, int64_t N, int64_t K, const void* A, int64_t sab,
                  int64_t sam, int64_t sak, const void* B, int64_t sbb, int64_t sbn, int64_t sbk, void* C, int64_t scb,
                  int64_t scm, int64_t scn) {
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  if (grid.y > 65535u) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "gemm: M too large for the native kernel");
  int ac = (sak == 1 || sam != 1) ? 0 : 1;
  int bc = (sbk == 1 || sbn != 1) ? 0 : 1;
  for (int64_t b0 = 0; b0 < nbatch; b0 += 65535) {
    grid.z = (unsigned)(nbatch - b0 < 65535 ? nbatch - b0 : 65535);
    const T* a = (const T*)A + b0 * sab;
    const T* b = (const T*)B + b0 * sbb;
    T* c = (T*)C + b0 * scb;
    if (ac == 0 && bc == 0)
      k_gemm_strided<T, 0, 0><<<grid, NT, 0, ctx->stream>>>(M, N, K, a, sam, sak, b, sbn, sbk, c, scm, scn, sab, sbb, scb);
    else if (ac == 0 && bc == 1)
      k_gemm_strided<T, 0, 1><<<grid, NT, 0, ctx->stream>>>(M, N, K, a, sam, sak, b, sbn, sbk, c, scm, scn, sab, sbb, scb);
    else if (ac == 1 && bc == 0)
      k_gemm_strided<T, 1, 0><<<grid, NT, 0, ctx->stream>>>(M, N, K, a, sam, sak, b, sbn, sbk, c, scm, scn, sab, sbb, scb);
    else
      k_gemm_strided<T, 1, 1><<<grid, NT, 0, ctx->stream>>>(M, N, K, a, sam, sak, b, sbn, sbk, c, scm, scn, sab, sbb, scb);
    TCI_CUDA(ctx, cudaGetLastError());
  }
  return TCI_OK;
}

}  // namespace

tci_status tci_gemm_native_batched(tci_context ctx, tci_dtype dt, int64_t nbatch, int64_t M, int64_t N, int64_t K,
                                   const void* A, int64_t sab, int64_t sam, int64_t sak, const void* B, int64_t sbb,
                                   int64_t sbn, int64_t sbk, void* C, int64_t scb, int64_t scm, int64_t scn) {
  if (nbatch <= 0 || M == 0 || N == 0) return TCI_OK;
  switch (dt) {
    case TCI_F32: return launch<float>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn);
    case TCI_F64: return launch<double>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn);
    case TCI_C64: return launch<float2>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn);
    case TCI_C128: return launch<double2>(ctx, nbatch, M, N, K, A, sab, sam, sak, B, sbb, sbn, sbk, C, scb, scm, scn);
  }
  return tci_fail(ctx, TCI_ERR_DTYPE, "gemm: bad dtype");
}

tci_status tci_gemm_native(tci_context ctx, tci_dtype dt, int64_t M, int64_t N, int64_t K, const void* A, int64_t sam,
                           int64_t sak, const void* B, int64_t sbn, int64_t sbk, void* C, int64_t scm, int64_t scn) {
  return tci_gemm_native_batched(ctx, dt, 1, M, N, K, A, 0, sam, sak, B, 0, sbn, sbk, C, 0, scm, scn);
}
