// Measured FP64 FMA rate of the device (a DFMA loop), the denominator of
// the FP64 rooflines.  The paper has no counterpart: its FP64 numbers come
// from other chips, and B300's FP64 rate is a small fraction of its tensor
// rate, so the FP64 paths are measured against what this chip sustains.
//
// Every thread runs kChains independent FMA chains a <- a * x + y with x, y
// read at run time (no constant folding); kChains chains hide the FMA
// latency.  One launch of kBlocksPerSM blocks per SM, `iters` iterations per
// chain; the result is stored so that no chain is dead code.
#include "tci_internal.cuh"

namespace {

constexpr int kProbeNT = 256;
constexpr int kChains = 8;
constexpr int kBlocksPerSM = 4;

__global__ void __launch_bounds__(kProbeNT) k_dfma_loop(const double* __restrict__ xy, int iters, double* __restrict__ sink) {
  const double x = xy[0], y = xy[1];
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" tci_status tci_probe_fp64_rate(tci_context ctx, int iters, double* gflops) {
  TCI_CHECK_CTX(ctx);
  if (!gflops || iters < 1) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "probe_fp64_rate: NULL output or iters < 1");
  const int blocks = ctx->num_sms * kBlocksPerSM;
  double* buf = nullptr;
  TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * ((size_t)blocks * kProbeNT + 2), (void**)&buf));
  // x slightly below 1 and y small keep every chain finite and normal
  const double xy[2] = {0.999999, 1e-7};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemcpyAsync(buf, xy, sizeof(xy), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
    e = cudaEventRecord(e0, ctx->stream);
    k_dfma_loop<<<blocks, kProbeNT, 0, ctx->stream>>>(buf, iters, buf + 2);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  tci_dev_free(buf);
  if (e != cudaSuccess) return tci_cuda_fail(ctx, e, "probe_fp64_rate");
  const double flops = 2.0 * kChains * (double)iters * blocks * kProbeNT;
  *gflops = best_ms > 0.f ? flops / (best_ms * 1e-3) / 1e9 : 0.0;
  return TCI_OK;
}
