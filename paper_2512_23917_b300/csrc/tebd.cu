// Batched two-site TEBD theta formation (the theta + gate step of the
// paper's iTEBD listing, App. A, batched over independent bonds):
//   theta_i[a, s1, s2, b] = sum_{t1, t2, c} G_i[s1, s2, t1, t2] A_i[a, t1, c] B_i[c, t2, b]
// complex64 in and out.  The complex product AB is ONE real split-BF16
// tensor-core GEMM per bond with the real and imaginary parts side by side:
//   rows (a, t1) = 2 chi:             A operand [Ar | Ai]            (depth 2 chi)
//   columns (b, t2, re) :             B operand [Br | -Bi]  -> Re AB
//   columns (b, t2, im) :             B operand [Bi |  Br]  -> Im AB
// so N = 4 chi and one output tile holds both t1 (adjacent rows = partner
// lanes), both t2 and both parts of 32 b.  The gate is the GEMM's epilogue
// (theta is formed in registers; AB never reaches memory), and all bonds run
// in ONE grouped persistent launch.  A split kernel before it builds the
// bfloat16 pieces (B transposed to K-major).
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tci_internal.cuh"

constexpr int kTebdMagic = 0x7ebd0001;

namespace {

int64_t pad8(int64_t x) { return (x + 7) / 8 * 8; }
// complex64 operands 8-byte aligned; G 16-byte aligned (the gate epilogue reads it as float4)
bool misaligned(const void* A, const void* B, const void* G, const void* theta) {
  return (((uintptr_t)A | (uintptr_t)B | (uintptr_t)theta) & 7) || ((uintptr_t)G & 15);
}
int64_t al256(int64_t bytes) { return (bytes + 255) / 256 * 256; }

struct BondJob {
  int64_t chi, Kh;                // Kh = pad8(chi): the depth of each half [re | im] of the K axis
  int64_t a_off, b_off, th_off;   // complex element offsets in the packed A, B, theta
  int64_t g_off;                  // complex element offset in the packed G (16 per bond)
  int64_t pa, pb;                 // bf16 element offsets (plane 0) of the A and B piece sets
};

// Pieces of 8 consecutive values: hi + mid + lo == x exactly (each residual is exact in FP32).
__device__ __forceinline__ void split8_store(__nv_bfloat16* base, int64_t plane, int64_t o, const float (&x)[8]) {
  uint4 w[3];
  uint32_t* h = reinterpret_cast<uint32_t*>(&w[0]);
  uint32_t* m = reinterpret_cast<uint32_t*>(&w[1]);
  uint32_t* l = reinterpret_cast<uint32_t*>(&w[2]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    const float2 hf = __bfloat1622float2(hh);
    const float r0 = x[2 * i] - hf.x, r1 = x[2 * i + 1] - hf.y;
    const __nv_bfloat162 mm = __floats2bfloat162_rn(r0, r1);
    const float2 mf = __bfloat1622float2(mm);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
    h[i] = *reinterpret_cast<const uint32_t*>(&hh);
    m[i] = *reinterpret_cast<const uint32_t*>(&mm);
    l[i] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  *reinterpret_cast<uint4*>(base + o) = w[0];
  *reinterpret_cast<uint4*>(base + plane + o) = w[1];
  *reinterpret_cast<uint4*>(base + 2 * plane + o) = w[2];
}

constexpr int kTQ = 32, kTC = 64;   // B transpose tile: 32 (t2, b) x 64 c

// Pieces of both operands of bond blockIdx.y (K axis [re half | im half], each
// half Kh deep, zero past chi), 8 consecutive k per thread (16-byte stores):
//   A rows (a, t1):      [Ar[a, t1, :] | Ai[a, t1, :]]
//   B rows (b, t2, re):  [Br[:, t2, b] | -Bi[:, t2, b]];  rows (b, t2, im): [Bi | Br]
// A is read along its contiguous c.  B goes through a shared-memory tile of
// 32 q = (t2, b) by 64 c: read with lanes along q (coalesced), written with 8
// lanes per output row (128 contiguous bytes per row and piece plane).  The
// first thread also publishes this call's gate and theta bases to gptr, where
// the GEMM's gate epilogue reads them (so a replayed graph patches this node only).
__global__ void __launch_bounds__(256) k_tebd_split(const BondJob* __restrict__ jobs, const float2* __restrict__ A,
                                                    const float2* __restrict__ B, __nv_bfloat16* __restrict__ arena,
                                                    const float2* G, float2* theta, const void** gptr) {
  __shared__ float2 tile[kTQ][kTC + 1];   // row length 65: lanes along q hit distinct bank pairs
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    gptr[0] = G;
    gptr[1] = theta;
  }
  const BondJob j = jobs[blockIdx.y];
  const int64_t chi = j.chi, Kh = j.Kh, Kp = 2 * Kh, nkc = Kh / 8, nq = 2 * chi;
  __nv_bfloat16* pa = arena + j.pa;
  const int64_t plane_a = 2 * chi * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 2 * chi * nkc;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / nkc, k0 = (e - r * nkc) * 8;
    float re[8], im[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 v = k0 + i < chi ? A[j.a_off + r * chi + k0 + i] : make_float2(0.f, 0.f);
      re[i] = v.x;
      im[i] = v.y;
    }
    split8_store(pa, plane_a, r * Kp + k0, re);
    split8_store(pa, plane_a, r * Kp + Kh + k0, im);
  }
  __nv_bfloat16* pb = arena + j.pb;
  const int64_t plane_b = 4 * chi * Kp;
  const int64_t ntc = (Kh + kTC - 1) / kTC, ntq = (nq + kTQ - 1) / kTQ;
  for (int64_t t = blockIdx.x; t < ntc * ntq; t += gridDim.x) {
    const int64_t c0 = (t % ntc) * kTC, q0 = (t / ntc) * kTQ;
    __syncthreads();   // the previous tile's readers are done
    for (int e = threadIdx.x; e < kTQ * kTC; e += blockDim.x) {
      const int ql = e % kTQ, cl = e / kTQ;
      const int64_t q = q0 + ql, c = c0 + cl;
      tile[ql][cl] = (q < nq && c < chi) ? B[j.b_off + c * nq + q] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int chunk = threadIdx.x % (kTC / 8), ql = threadIdx.x / (kTC / 8);   // 8 x 32 items
    const int64_t q = q0 + ql, k0 = c0 + chunk * 8;
    if (q < nq && k0 < Kh) {
      float re[8], im[8], nim[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 v = tile[ql][chunk * 8 + i];
        re[i] = v.x;
        im[i] = v.y;
        nim[i] = -v.y;
      }
      const int64_t t2 = q / chi, b = q - t2 * chi;
      const int64_t n = (b * 2 + t2) * 2;   // row (b, t2, re); (b, t2, im) follows
      split8_store(pb, plane_b, n * Kp + k0, re);
      split8_store(pb, plane_b, n * Kp + Kh + k0, nim);
      split8_store(pb, plane_b, (n + 1) * Kp + k0, im);
      split8_store(pb, plane_b, (n + 1) * Kp + Kh + k0, re);
    }
  }
}

}  // namespace

struct tci_tebd_plan_s {
  int magic;
  tci_context ctx;
  int nbonds;
  int products, chunk_k, xchunk_k;
  int raster = 0;
  int64_t max_chi;
  double flops;
  double tensor_flops = 0.0;
  void* arena = nullptr;   // bf16 pieces
  BondJob* d_jobs = nullptr;
  const void** d_gptr = nullptr;   // {gate base, theta base} of the current call
  tci_split_group* group = nullptr;    // 128-wide tiles
  tci_split_group* group_n = nullptr;  // 64-wide tiles (a tile shape the autotuner may choose)
  int bn = 128;
  tci_graph graph;   // captured split -> grouped GEMM (gate epilogue)
  const void *cA = nullptr, *cB = nullptr, *cG = nullptr;
  void* cT = nullptr;
};

extern "C" tci_status tci_tebd_plan_destroy(tci_tebd_plan* pp) {
  if (!pp || !*pp || (*pp)->magic != kTebdMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "tebd_plan_destroy: invalid plan");
  tci_tebd_plan p = *pp;
  if (tci_ctx_ok(p->ctx)) cudaStreamSynchronize(p->ctx->stream);
  tci_graph_destroy(&p->graph);
  tci_split_group_destroy(p->group);
  tci_split_group_destroy(p->group_n);
  tci_dev_free(p->arena);
  tci_dev_free(p->d_jobs);
  tci_dev_free(p->d_gptr);
  p->magic = 0;
  delete p;
  *pp = nullptr;
  return TCI_OK;
}

extern "C" tci_status tci_tebd_plan_create(tci_context ctx, int nbonds, const int64_t* chi, tci_tebd_plan* out) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "tebd_plan_create");
  if (!out) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_plan_create: NULL output");
  *out = nullptr;
  if (nbonds <= 0 || !chi) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_plan_create: no bonds");
  if (ctx->precision == TCI_PREC_NATIVE)
    return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "tebd_plan_create: the batched theta path runs in a split precision");
  tci_tebd_plan p = new tci_tebd_plan_s();
  p->magic = kTebdMagic;
  p->ctx = ctx;
  p->nbonds = nbonds;
  p->products = ctx->precision == TCI_PREC_SPLIT_BF16_3 ? 3 : 6;
  p->chunk_k = ctx->split_chunk_k;
  p->xchunk_k = ctx->split_xchunk_k;
  p->max_chi = 0;
  auto fail = [&](tci_status s) {
    tci_tebd_plan pp = p;
    tci_tebd_plan_destroy(&pp);
    return s;
  };
  std::vector<BondJob> jobs(nbonds);
  int64_t arena = 0, aoff = 0, thoff = 0;
  double fl = 0.0;
  for (int i = 0; i < nbonds; ++i) {
    if (chi[i] <= 0) return fail(tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_plan_create: bond %d has chi %lld", i, (long long)chi[i]));
    BondJob& j = jobs[i];
    j.chi = chi[i];
    j.Kh = pad8(j.chi);
    j.a_off = aoff;
    j.b_off = aoff;
    j.th_off = thoff;
    j.g_off = 16 * (int64_t)i;
    aoff += 2 * j.chi * j.chi;
    thoff += 4 * j.chi * j.chi;
    const int64_t Kp = 2 * j.Kh;
    j.pa = arena;
    arena += al256(3 * 2 * j.chi * Kp * 2) / 2;
    j.pb = arena;
    arena += al256(3 * 4 * j.chi * Kp * 2) / 2;
    p->max_chi = std::max(p->max_chi, j.chi);
    const double c = (double)j.chi;
    fl += 8.0 * c * c * c * 4.0 + 8.0 * c * c * 16.0;   // 8 chi^3 d^2 + 8 chi^2 d^4
    p->tensor_flops += 2.0 * p->products * (2.0 * c) * (4.0 * c) * (double)Kp;
  }
  p->flops = fl;
  tci_status s;
  if ((s = tci_dev_alloc(ctx, arena * 2, &p->arena)) != TCI_OK) return fail(s);
  if ((s = tci_dev_alloc(ctx, sizeof(BondJob) * nbonds, (void**)&p->d_jobs)) != TCI_OK) return fail(s);
  if ((s = tci_dev_alloc(ctx, 2 * sizeof(void*), (void**)&p->d_gptr)) != TCI_OK) return fail(s);
  cudaError_t e = cudaMemcpyAsync(p->d_jobs, jobs.data(), sizeof(BondJob) * nbonds, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "tebd plan: jobs"));
  std::vector<tci_split_problem> probs;
  __nv_bfloat16* A = (__nv_bfloat16*)p->arena;
  for (int i = 0; i < nbonds; ++i) {
    const BondJob& j = jobs[i];
    tci_split_problem q = {A + j.pa, A + j.pb, 2 * j.chi, 4 * j.chi, 2 * j.Kh, nullptr, 3, 0, 0};
    q.g_chi = j.chi;
    q.g_off = j.g_off;
    q.th_off = j.th_off;
    probs.push_back(q);
  }
  if ((s = tci_split_group_create(ctx, (int)probs.size(), probs.data(), &p->group, 128)) != TCI_OK) return fail(s);
  if ((s = tci_split_group_create(ctx, (int)probs.size(), probs.data(), &p->group_n, 64)) != TCI_OK) return fail(s);
  vs.info = "bonds=" + std::to_string(nbonds) + " max_chi=" + std::to_string(p->max_chi);
  *out = p;
  return TCI_OK;
}

extern "C" double tci_tebd_flops(tci_tebd_plan p) {
  if (!p || p->magic != kTebdMagic) return 0.0;
  return p->flops;
}

// one block row per bond; up to 64 blocks per bond (the largest bond's B
// tiles of 32 x 64, or its A pass in items of 8 by blocks of 256)
static dim3 split_grid(const tci_tebd_plan_s* p) {
  const int64_t mc = p->max_chi;
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (2 * mc * pad8(mc) / 8 + 255) / 256)), (unsigned)p->nbonds);
}

static tci_status tebd_launch_all(void* arg) {
  tci_tebd_plan p = (tci_tebd_plan)arg;
  tci_context ctx = p->ctx;
  k_tebd_split<<<split_grid(p), 256, 0, ctx->stream>>>(p->d_jobs, (const float2*)p->cA, (const float2*)p->cB,
                                                       (__nv_bfloat16*)p->arena, (const float2*)p->cG,
                                                       (float2*)p->cT, p->d_gptr);
  TCI_CUDA(ctx, cudaGetLastError());
  return tci_split_group_launch(ctx, p->bn == 64 ? p->group_n : p->group, p->products, p->chunk_k, p->xchunk_k,
                                p->raster, (const void* const*)p->d_gptr);
}

extern "C" tci_status tci_tebd_apply(tci_tebd_plan p, const void* A, const void* B, const void* G, void* theta) {
  if (!p || p->magic != kTebdMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "tebd_apply: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "tebd_apply");
  if (!A || !B || !G || !theta) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_apply: NULL buffer");
  if (misaligned(A, B, G, theta)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_apply: misaligned buffer");
  p->cA = A;
  p->cB = B;
  p->cG = G;
  p->cT = theta;
  if (!p->graph.exec) {
    TCI_TRY(tebd_launch_all(p));
    return tci_graph_capture(ctx, &p->graph, tebd_launch_all, p, {(const void*)k_tebd_split});
  }
  const BondJob* jobs = p->d_jobs;
  __nv_bfloat16* arena = (__nv_bfloat16*)p->arena;
  const void** gptr = p->d_gptr;
  void* sargs[7] = {(void*)&jobs, (void*)&A, (void*)&B, (void*)&arena, (void*)&G, (void*)&theta, (void*)&gptr};
  cudaKernelNodeParams kp;
  TCI_CUDA(ctx, cudaGraphKernelNodeGetParams(p->graph.nodes[0], &kp));
  kp.kernelParams = sargs;
  kp.extra = nullptr;
  TCI_CUDA(ctx, cudaGraphExecKernelNodeSetParams(p->graph.exec, p->graph.nodes[0], &kp));
  TCI_CUDA(ctx, cudaGraphLaunch(p->graph.exec, ctx->stream));
  return TCI_OK;
}

// tci_tebd_apply with CUDA events between the stages: ms[0] = split, ms[1] =
// grouped GEMM (one per bond, gate in its epilogue), ms[2] = 0
// (no separate gate stage).  Synchronises.
extern "C" tci_status tci_tebd_apply_timed(tci_tebd_plan p, const void* A, const void* B, const void* G, void* theta,
                                           float* ms) {
  if (!p || p->magic != kTebdMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "tebd_apply_timed: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  if (!A || !B || !G || !theta || !ms) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_apply_timed: NULL argument");
  if (misaligned(A, B, G, theta)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_apply_timed: misaligned buffer");
  cudaEvent_t ev[3];
  for (auto& e : ev) TCI_CUDA(ctx, cudaEventCreate(&e));
  TCI_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream));
  k_tebd_split<<<split_grid(p), 256, 0, ctx->stream>>>(p->d_jobs, (const float2*)A, (const float2*)B,
                                                       (__nv_bfloat16*)p->arena, (const float2*)G, (float2*)theta,
                                                       p->d_gptr);
  TCI_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
  TCI_TRY(tci_split_group_launch(ctx, p->bn == 64 ? p->group_n : p->group, p->products, p->chunk_k, p->xchunk_k,
                                 p->raster, (const void* const*)p->d_gptr));
  TCI_CUDA(ctx, cudaEventRecord(ev[2], ctx->stream));
  TCI_CUDA(ctx, cudaEventSynchronize(ev[2]));
  for (int i = 0; i < 2; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  ms[2] = 0.f;
  for (auto& e : ev) cudaEventDestroy(e);
  return tci_synchronize(ctx);
}

// BF16 tensor flops executed by the grouped launch: one real GEMM per bond,
// 2 * products * (2 chi) * (4 chi) * 2 pad8(chi).
extern "C" double tci_tebd_tensor_flops(tci_tebd_plan p) {
  if (!p || p->magic != kTebdMagic) return 0.0;
  return p->tensor_flops;
}

// ---------------------------------------------------------------- autotuning
namespace {
tci_status tebd_run_cfg(void* a, const tci_gemm_cfg& cfg) {
  tci_tebd_plan p = (tci_tebd_plan)a;
  p->chunk_k = cfg.chunk_k;
  p->xchunk_k = cfg.xchunk_k;
  p->raster = cfg.raster;
  p->bn = cfg.bn;
  return tebd_launch_all(p);
}
}  // namespace

extern "C" tci_status tci_tebd_autotune(tci_tebd_plan p, const void* A, const void* B, const void* G, void* theta,
                                        int max_chunk_k, int* chosen) {
  if (!p || p->magic != kTebdMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "tebd_autotune: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "tebd_autotune");
  if (!A || !B || !G || !theta) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_autotune: NULL buffer");
  if (misaligned(A, B, G, theta)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_autotune: misaligned buffer");
  p->cA = A;
  p->cB = B;
  p->cG = G;
  p->cT = theta;
  const std::string key = "tebd|b" + std::to_string(p->nbonds) + "|max" + std::to_string(p->max_chi) + "|f" +
                          std::to_string((long long)(p->flops / 1e6)) + "|p" + std::to_string(p->products);
  tci_gemm_cfg best;
  double ms = 0.0;
  TCI_TRY(tci_autotune(ctx, key, max_chunk_k, true, tebd_run_cfg, p, &best, &ms, true));
  p->chunk_k = best.chunk_k;
  p->xchunk_k = best.xchunk_k;
  p->raster = best.raster;
  p->bn = best.bn;
  tci_graph_destroy(&p->graph);
  if (chosen) {
    chosen[0] = best.chunk_k;
    chosen[1] = best.xchunk_k;
    chosen[2] = best.raster;
  }
  return tci_synchronize(ctx);
}

// ------------------------------------------------------------------ handle form
extern "C" tci_status tci_tebd_theta_batched(tci_context ctx, int n, const tci_tensor* A, const tci_tensor* B,
                                             const tci_tensor* G, tci_tensor* theta) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "tebd_theta_batched");
  if (n < 0 || (n > 0 && (!A || !B || !G || !theta)))
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_theta_batched: invalid arrays");
  if (n == 0) return TCI_OK;
  std::vector<int64_t> chi(n);
  for (int i = 0; i < n; ++i) {
    const tci_tensor a = A[i], b = B[i], g = G[i];
    if (!tci_ten_ok(a) || !tci_ten_ok(b) || !tci_ten_ok(g))
      return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_theta_batched: invalid tensor of bond %d", i);
    if (a->dtype != TCI_C64 || b->dtype != TCI_C64 || g->dtype != TCI_C64)
      return tci_fail(ctx, TCI_ERR_DTYPE, "tebd_theta_batched: A, B, G must be C64 (bond %d)", i);
    const int64_t c = a->order == 3 ? a->shape[0] : -1;
    if (c < 1 || a->shape[1] != 2 || a->shape[2] != c || b->order != 3 || b->shape[0] != c || b->shape[1] != 2 ||
        b->shape[2] != c || g->order != 4 || g->shape[0] != 2 || g->shape[1] != 2 || g->shape[2] != 2 ||
        g->shape[3] != 2 || !tci_is_rowmajor(a) || !tci_is_rowmajor(b) || !tci_is_rowmajor(g))
      return tci_fail(ctx, TCI_ERR_SHAPE, "tebd_theta_batched: bond %d needs row-major A, B [chi,2,chi], G [2,2,2,2]", i);
    if (theta[i]) {
      const tci_tensor t = theta[i];
      if (!tci_ten_ok(t) || t->dtype != TCI_C64 || t->order != 4 || t->shape[0] != c || t->shape[1] != 2 ||
          t->shape[2] != 2 || t->shape[3] != c || !tci_is_rowmajor(t))
        return tci_fail(ctx, TCI_ERR_SHAPE, "tebd_theta_batched: theta of bond %d must be C64 [chi,2,2,chi]", i);
    }
    chi[i] = c;
  }
  tci_tebd_plan plan = nullptr;
  TCI_TRY(tci_tebd_plan_create(ctx, n, chi.data(), &plan));
  int64_t na = 0, nt = 0;
  for (int64_t c : chi) {
    na += 2 * c * c;
    nt += 4 * c * c;
  }
  const size_t eb = 2 * sizeof(float);
  void *pa = nullptr, *pb = nullptr, *pg = nullptr, *pt = nullptr;
  tci_status st = tci_dev_alloc(ctx, eb * na, &pa);
  if (st == TCI_OK) st = tci_dev_alloc(ctx, eb * na, &pb);
  if (st == TCI_OK) st = tci_dev_alloc(ctx, eb * 16 * n, &pg);
  if (st == TCI_OK) st = tci_dev_alloc(ctx, eb * nt, &pt);
  cudaError_t e = cudaSuccess;
  int64_t oa = 0, ot = 0;
  for (int i = 0; i < n && st == TCI_OK && e == cudaSuccess; ++i) {
    const int64_t c = chi[i];
    e = cudaMemcpyAsync((char*)pa + eb * oa, A[i]->data, eb * 2 * c * c, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char*)pb + eb * oa, B[i]->data, eb * 2 * c * c, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char*)pg + eb * 16 * i, G[i]->data, eb * 16, cudaMemcpyDeviceToDevice, ctx->stream);
    oa += 2 * c * c;
  }
  if (st == TCI_OK && e != cudaSuccess) st = tci_cuda_fail(ctx, e, "tebd_theta_batched: pack");
  if (st == TCI_OK) st = tci_tebd_apply(plan, pa, pb, pg, pt);
  for (int i = 0; i < n && st == TCI_OK; ++i) {
    const int64_t c = chi[i];
    if (!theta[i]) {
      const int64_t shp[4] = {c, 2, 2, c};
      st = tci_allocate(ctx, TCI_C64, 4, shp, &theta[i]);
      if (st != TCI_OK) break;
    }
    e = cudaMemcpyAsync(theta[i]->data, (char*)pt + eb * ot, eb * 4 * c * c, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) st = tci_cuda_fail(ctx, e, "tebd_theta_batched: unpack");
    ot += 4 * c * c;
  }
  if (st == TCI_OK) st = tci_synchronize(ctx);
  for (void* q : {pa, pb, pg, pt}) tci_dev_free(q);
  tci_tebd_plan_destroy(&plan);
  return st;
}

extern "C" tci_status tci_tebd_set_tile_n(tci_tebd_plan p, int bn) {
  if (!p || p->magic != kTebdMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "tebd_set_tile_n: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  if (bn != 64 && bn != 128) return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "tebd_set_tile_n: tile width 64 or 128");
  if (bn != p->bn) {
    cudaStreamSynchronize(p->ctx->stream);
    tci_graph_destroy(&p->graph);   // the next apply captures the new sequence
    p->bn = bn;
  }
  return TCI_OK;
}

extern "C" int tci_tebd_tile_n(tci_tebd_plan p) {
  if (!p || p->magic != kTebdMagic) return -1;
  return p->bn;
}
