// Allocation-free FP64 two-site H_eff matvec for small bond dimensions.
//
// Who needs this: code that must not allocate GPU memory at the point where
// it applies H_eff -- for example a caller running under a memory manager
// that owns every byte of the device, a real-time loop that forbids
// cudaMalloc/cudaFree (they synchronise the device), or a host whose
// allocator is not available.  The regular path (tci_heff_plan_create +
// tci_heff_apply) allocates its intermediates once per plan; this entry
// point instead keeps them in one fixed array compiled into the library.
//
// Scratch: `g_heff_noalloc_scratch`, TCI_HEFF_NOALLOC_SCRATCH_DOUBLES
// doubles (4 MiB) of device memory, present on every GPU that loads the
// library until the process exits.  A call needs 512 + 40 * chiL * chiR
// doubles (a 512-double slot for the W.W table, then the U and V
// intermediates), so chiL * chiR <= 13094 (e.g. chi = 114 on both sides);
// larger requests are rejected before anything is launched.
//
// Every call reuses the same array, so two calls whose kernels overlap on
// the GPU (different streams, or different host threads on one device)
// race and produce garbage; serialise them.  Each call writes every scratch
// element it later reads before reading it, so stale contents from the
// previous call never matter and nothing needs clearing.
//
// The device address of the array is looked up with cudaGetSymbolAddress
// the first time the entry point runs on a device (with that device
// current), and cached per device; make that first call before starting
// any stream capture on the device.
#include <mutex>

#include "tci_internal.cuh"

#define TCI_HEFF_NOALLOC_SCRATCH_DOUBLES (1 << 19)

static __device__ __align__(256) double g_heff_noalloc_scratch[TCI_HEFF_NOALLOC_SCRATCH_DOUBLES];

namespace {

constexpr int kDw = 5;
constexpr int kD = 2;
constexpr int kNWW = kDw * kD * kD * kDw * kD * kD;   // 400
constexpr int kMaxDevices = 64;

// WW[wl][s1][s2][wr][t1][t2] = sum_wm W[wl,wm,s1,t1] W[wm,wr,s2,t2]
__global__ void k_na_ww(const double* __restrict__ W, double* __restrict__ WW) {
  for (int i = threadIdx.x; i < kNWW; i += blockDim.x) {
    int r = i;
    const int t2 = r % kD; r /= kD;
    const int t1 = r % kD; r /= kD;
    const int wr = r % kDw; r /= kDw;
    const int s2 = r % kD; r /= kD;
    const int s1 = r % kD; r /= kD;
    const int wl = r;
    double acc = 0.0;
    for (int wm = 0; wm < kDw; ++wm)
      acc += W[((wl * kDw + wm) * kD + s1) * kD + t1] * W[((wm * kDw + wr) * kD + s2) * kD + t2];
    WW[i] = acc;
  }
}

// C[m*ldc + n] = sum_k A[m*lda + k] B[n*ldb + k]   (one thread per output)
__global__ void k_na_gemm_tn(int64_t M, int64_t N, int64_t K, const double* __restrict__ A, int64_t lda,
                             const double* __restrict__ B, int64_t ldb, double* __restrict__ C, int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = i / N, n = i - m * N;
    double acc = 0.0;
    for (int64_t k = 0; k < K; ++k) acc = fma(A[m * lda + k], B[n * ldb + k], acc);
    C[m * ldc + n] = acc;
  }
}

// V[(s1 s2, b), (wl, a')] = sum_{wr, t1 t2} WW[wl][s][wr][t] U[(a', t), (b, wr)]
__global__ void k_na_ww_apply(const double* __restrict__ WW, const double* __restrict__ U, int64_t chiL, int64_t chiR,
                              double* __restrict__ V) {
  const int64_t total = chiL * chiR;
  const int64_t ldu = chiR * kDw, ldv = kDw * chiL;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ap = i / chiR, b = i - ap * chiR;
    double in[4 * kDw];
    for (int t = 0; t < 4; ++t)
      for (int wr = 0; wr < kDw; ++wr) in[t * kDw + wr] = U[(ap * 4 + t) * ldu + b * kDw + wr];
    for (int wl = 0; wl < kDw; ++wl)
      for (int s = 0; s < 4; ++s) {
        double acc = 0.0;
        for (int wr = 0; wr < kDw; ++wr)
          for (int t = 0; t < 4; ++t) acc = fma(WW[((wl * 4 + s) * kDw + wr) * 4 + t], in[t * kDw + wr], acc);
        V[(s * chiR + b) * ldv + wl * chiL + ap] = acc;
      }
  }
}

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

int grid_for(int64_t work) {
  int64_t b = (work + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

extern "C" tci_status tci_heff_apply_noalloc(const double* L, const double* W, const double* R, const double* psi,
                                             double* out, int64_t chiL, int64_t chiR, void* stream) {
  if (!L || !W || !R || !psi || !out) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_apply_noalloc: NULL pointer");
  if (chiL <= 0 || chiR <= 0) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_apply_noalloc: bond dimensions must be positive");
  if (chiL > TCI_HEFF_NOALLOC_SCRATCH_DOUBLES || chiR > TCI_HEFF_NOALLOC_SCRATCH_DOUBLES ||
      512 + 40 * chiL * chiR > (int64_t)TCI_HEFF_NOALLOC_SCRATCH_DOUBLES)
    return tci_fail(nullptr, TCI_ERR_UNSUPPORTED,
                    "heff_apply_noalloc: chiL*chiR = %lld exceeds the fixed scratch (needs 512 + 40*chiL*chiR <= %d doubles, "
                    "i.e. chiL*chiR <= 13094); use tci_heff_plan_create/tci_heff_apply",
                    (long long)(chiL * chiR), TCI_HEFF_NOALLOC_SCRATCH_DOUBLES);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tci_cuda_fail(nullptr, e, "heff_apply_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return tci_fail(nullptr, TCI_ERR_UNSUPPORTED, "heff_apply_noalloc: device index %d", dev);
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_heff_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return tci_cuda_fail(nullptr, e, "heff_apply_noalloc: cudaGetSymbolAddress");
      g_scratch_addr[dev] = (double*)ptr;
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* WW = scratch;                              // 400 doubles (512 reserved)
  double* U = scratch + 512;                         // [(a', t), (b, wr)]  chiL*4 x chiR*5
  double* V = U + 20 * chiL * chiR;                  // [(s, b), (wl, a')]  4*chiR x 5*chiL
  k_na_ww<<<1, 256, 0, st>>>(W, WW);
  k_na_gemm_tn<<<grid_for(chiL * 4 * chiR * kDw), 256, 0, st>>>(chiL * 4, chiR * kDw, chiR, psi, chiR, R, chiR, U,
                                                                 chiR * kDw);
  k_na_ww_apply<<<grid_for(chiL * chiR), 256, 0, st>>>(WW, U, chiL, chiR, V);
  k_na_gemm_tn<<<grid_for(chiL * 4 * chiR), 256, 0, st>>>(chiL, 4 * chiR, kDw * chiL, L, kDw * chiL, V, kDw * chiL, out,
                                                          4 * chiR);
  e = cudaGetLastError();
  if (e != cudaSuccess) return tci_cuda_fail(nullptr, e, "heff_apply_noalloc: launch");
  return TCI_OK;
}
