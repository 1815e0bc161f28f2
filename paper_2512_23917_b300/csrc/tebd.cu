// Batched two-site TEBD theta formation (the theta + gate step of the
// paper's iTEBD listing, App. A, batched over independent bonds):
//   theta_i[a, s1, s2, b] = sum_{t1, t2, c} G_i[s1, s2, t1, t2] A_i[a, t1, c] B_i[c, t2, b]
// complex64 in and out.  The complex product AB uses three real products
// (3M):  P1 = Ar Br,  P2 = Ai Bi,  P3 = (Ar + Ai)(Br + Bi);
//        Re AB = P1 - P2,  Im AB = P3 - P1 - P2.
// Each real product is a split-BF16 tensor-core GEMM with
//   rows (a, t1) = 2 chi, columns (t2, b) = 2 chi, depth c = chi;
// all 3 x nbonds GEMMs run in ONE grouped persistent launch.  A split
// kernel before it builds the bfloat16 pieces (B is transposed to K-major
// while it is split), and a gate kernel after it applies G.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tci_internal.cuh"

constexpr int kTebdMagic = 0x7ebd0001;

namespace {

int64_t pad8(int64_t x) { return (x + 7) / 8 * 8; }
int64_t al256(int64_t bytes) { return (bytes + 255) / 256 * 256; }

struct BondJob {
  int64_t chi, Kp;
  int64_t a_off, b_off, th_off;   // complex element offsets in the packed A, B, theta
  int64_t g_off;                  // complex element offset in the packed G (16 per bond)
  int64_t pa[3], pb[3];           // bf16 element offsets (plane 0) of the 3 operand piece sets
  int64_t pc[3];                  // float offsets of P1, P2, P3 ([2chi][2chi])
};

__device__ __forceinline__ void split_store(__nv_bfloat16* base, int64_t plane, int64_t o, float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
  base[o] = h;
  base[plane + o] = m;
  base[2 * plane + o] = l;
}

// A_i as [(a, t1), c] (already K-major) and B_i^T as [(t2, b), c]; each split
// into the pieces of its real part, imaginary part and real + imaginary.
__global__ void k_tebd_split(const BondJob* __restrict__ jobs, const float2* __restrict__ A,
                             const float2* __restrict__ B, __nv_bfloat16* __restrict__ arena) {
  const BondJob j = jobs[blockIdx.y];
  const int64_t rows = 2 * j.chi, K = j.chi, Kp = j.Kp, plane = rows * Kp;
  const int64_t n = rows * Kp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / Kp, k = i - r * Kp;
    float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
    if (k < K) {
      va = A[j.a_off + r * K + k];                 // A[a, t1, c] with r = (a, t1)
      vb = B[j.b_off + k * rows + r];              // B[c, t2, b] with r = (t2, b)
    }
    split_store(arena + j.pa[0], plane, i, va.x);
    split_store(arena + j.pa[1], plane, i, va.y);
    split_store(arena + j.pa[2], plane, i, va.x + va.y);
    split_store(arena + j.pb[0], plane, i, vb.x);
    split_store(arena + j.pb[1], plane, i, vb.y);
    split_store(arena + j.pb[2], plane, i, vb.x + vb.y);
  }
}

// theta[a, s1, s2, b] = sum_{t1,t2} G[s1,s2,t1,t2] AB[(a,t1),(t2,b)]
__global__ void k_tebd_gate(const BondJob* __restrict__ jobs, const float* __restrict__ P, const float2* __restrict__ G,
                            float2* __restrict__ theta) {
  const BondJob j = jobs[blockIdx.y];
  const int64_t chi = j.chi, ld = 2 * chi;
  float2 g[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) g[q] = G[j.g_off + q];
  const float* P1 = P + j.pc[0];
  const float* P2 = P + j.pc[1];
  const float* P3 = P + j.pc[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < chi * chi; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / chi, b = i - a * chi;
    float2 ab[4];
#pragma unroll
    for (int t1 = 0; t1 < 2; ++t1)
#pragma unroll
      for (int t2 = 0; t2 < 2; ++t2) {
        const int64_t o = (2 * a + t1) * ld + t2 * chi + b;
        const float p1 = P1[o], p2 = P2[o], p3 = P3[o];
        ab[t1 * 2 + t2] = make_float2(p1 - p2, p3 - p1 - p2);
      }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float2 gg = g[s * 4 + t];
        re = fmaf(gg.x, ab[t].x, fmaf(-gg.y, ab[t].y, re));
        im = fmaf(gg.x, ab[t].y, fmaf(gg.y, ab[t].x, im));
      }
      theta[j.th_off + (a * 4 + s) * chi + b] = make_float2(re, im);
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
  float* P = nullptr;      // P1, P2, P3 per bond
  BondJob* d_jobs = nullptr;
  tci_split_group* group = nullptr;    // 128-wide tiles
  tci_split_group* group_n = nullptr;  // 64-wide tiles (a tile shape the autotuner may choose)
  int bn = 128;
  tci_graph graph;   // captured split -> grouped GEMM -> gate
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
  tci_dev_free(p->P);
  tci_dev_free(p->d_jobs);
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
  int64_t arena = 0, pels = 0, aoff = 0, thoff = 0;
  double fl = 0.0;
  for (int i = 0; i < nbonds; ++i) {
    if (chi[i] <= 0) return fail(tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_plan_create: bond %d has chi %lld", i, (long long)chi[i]));
    BondJob& j = jobs[i];
    j.chi = chi[i];
    j.Kp = pad8(j.chi);
    j.a_off = aoff;
    j.b_off = aoff;
    j.th_off = thoff;
    j.g_off = 16 * (int64_t)i;
    aoff += 2 * j.chi * j.chi;
    thoff += 4 * j.chi * j.chi;
    const int64_t piece_elems = al256(3 * 2 * j.chi * j.Kp * 2) / 2;
    for (int q = 0; q < 3; ++q) {
      j.pa[q] = arena;
      arena += piece_elems;
    }
    for (int q = 0; q < 3; ++q) {
      j.pb[q] = arena;
      arena += piece_elems;
    }
    for (int q = 0; q < 3; ++q) {
      j.pc[q] = pels;
      pels += al256(4 * j.chi * j.chi * 4) / 4;
    }
    p->max_chi = std::max(p->max_chi, j.chi);
    const double c = (double)j.chi;
    fl += 8.0 * c * c * c * 4.0 + 8.0 * c * c * 16.0;   // 8 chi^3 d^2 + 8 chi^2 d^4
    p->tensor_flops += 3.0 * 2.0 * p->products * (2.0 * c) * (2.0 * c) * (double)j.Kp;
  }
  p->flops = fl;
  tci_status s;
  if ((s = tci_dev_alloc(ctx, arena * 2, &p->arena)) != TCI_OK) return fail(s);
  if ((s = tci_dev_alloc(ctx, pels * 4, (void**)&p->P)) != TCI_OK) return fail(s);
  if ((s = tci_dev_alloc(ctx, sizeof(BondJob) * nbonds, (void**)&p->d_jobs)) != TCI_OK) return fail(s);
  cudaError_t e = cudaMemcpyAsync(p->d_jobs, jobs.data(), sizeof(BondJob) * nbonds, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "tebd plan: jobs"));
  std::vector<tci_split_problem> probs;
  __nv_bfloat16* A = (__nv_bfloat16*)p->arena;
  for (int i = 0; i < nbonds; ++i) {
    const BondJob& j = jobs[i];
    for (int q = 0; q < 3; ++q)
      probs.push_back({A + j.pa[q], A + j.pb[q], 2 * j.chi, 2 * j.chi, j.Kp, p->P + j.pc[q], 1, 2 * j.chi, 1});
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

static tci_status tebd_launch_all(void* arg) {
  tci_tebd_plan p = (tci_tebd_plan)arg;
  tci_context ctx = p->ctx;
  const int64_t mc = p->max_chi;
  dim3 g1((unsigned)std::max<int64_t>(1, std::min<int64_t>(128, (2 * mc * pad8(mc) + 255) / 256)), (unsigned)p->nbonds);
  k_tebd_split<<<g1, 256, 0, ctx->stream>>>(p->d_jobs, (const float2*)p->cA, (const float2*)p->cB, (__nv_bfloat16*)p->arena);
  TCI_CUDA(ctx, cudaGetLastError());
  TCI_TRY(tci_split_group_launch(ctx, p->bn == 64 ? p->group_n : p->group, p->products, p->chunk_k, p->xchunk_k,
                                 p->raster));
  dim3 g2((unsigned)std::max<int64_t>(1, std::min<int64_t>(128, (mc * mc + 255) / 256)), (unsigned)p->nbonds);
  k_tebd_gate<<<g2, 256, 0, ctx->stream>>>(p->d_jobs, p->P, (const float2*)p->cG, (float2*)p->cT);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

extern "C" tci_status tci_tebd_apply(tci_tebd_plan p, const void* A, const void* B, const void* G, void* theta) {
  if (!p || p->magic != kTebdMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "tebd_apply: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "tebd_apply");
  if (!A || !B || !G || !theta) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_apply: NULL buffer");
  p->cA = A;
  p->cB = B;
  p->cG = G;
  p->cT = theta;
  if (!p->graph.exec) {
    TCI_TRY(tebd_launch_all(p));
    return tci_graph_capture(ctx, &p->graph, tebd_launch_all, p, {(const void*)k_tebd_split, (const void*)k_tebd_gate});
  }
  const BondJob* jobs = p->d_jobs;
  __nv_bfloat16* arena = (__nv_bfloat16*)p->arena;
  const float* P = p->P;
  void* sargs[4] = {(void*)&jobs, (void*)&A, (void*)&B, (void*)&arena};
  void* gargs[4] = {(void*)&jobs, (void*)&P, (void*)&G, (void*)&theta};
  void** argv[2] = {sargs, gargs};
  for (int i = 0; i < 2; ++i) {
    cudaKernelNodeParams kp;
    TCI_CUDA(ctx, cudaGraphKernelNodeGetParams(p->graph.nodes[i], &kp));
    kp.kernelParams = argv[i];
    kp.extra = nullptr;
    TCI_CUDA(ctx, cudaGraphExecKernelNodeSetParams(p->graph.exec, p->graph.nodes[i], &kp));
  }
  TCI_CUDA(ctx, cudaGraphLaunch(p->graph.exec, ctx->stream));
  return TCI_OK;
}

// tci_tebd_apply with CUDA events between the stages: ms[0..2] = split,
// grouped GEMM (3 real products per bond), gate.  Synchronises.
extern "C" tci_status tci_tebd_apply_timed(tci_tebd_plan p, const void* A, const void* B, const void* G, void* theta,
                                           float* ms) {
  if (!p || p->magic != kTebdMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "tebd_apply_timed: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  if (!A || !B || !G || !theta || !ms) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "tebd_apply_timed: NULL argument");
  cudaEvent_t ev[4];
  for (auto& e : ev) TCI_CUDA(ctx, cudaEventCreate(&e));
  const int64_t mc = p->max_chi;
  TCI_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream));
  dim3 g1((unsigned)std::max<int64_t>(1, std::min<int64_t>(128, (2 * mc * pad8(mc) + 255) / 256)), (unsigned)p->nbonds);
  k_tebd_split<<<g1, 256, 0, ctx->stream>>>(p->d_jobs, (const float2*)A, (const float2*)B, (__nv_bfloat16*)p->arena);
  TCI_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
  TCI_TRY(tci_split_group_launch(ctx, p->bn == 64 ? p->group_n : p->group, p->products, p->chunk_k, p->xchunk_k,
                                 p->raster));
  TCI_CUDA(ctx, cudaEventRecord(ev[2], ctx->stream));
  dim3 g2((unsigned)std::max<int64_t>(1, std::min<int64_t>(128, (mc * mc + 255) / 256)), (unsigned)p->nbonds);
  k_tebd_gate<<<g2, 256, 0, ctx->stream>>>(p->d_jobs, p->P, (const float2*)G, (float2*)theta);
  TCI_CUDA(ctx, cudaEventRecord(ev[3], ctx->stream));
  TCI_CUDA(ctx, cudaEventSynchronize(ev[3]));
  for (int i = 0; i < 3; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  for (auto& e : ev) cudaEventDestroy(e);
  return tci_synchronize(ctx);
}

// BF16 tensor flops executed by the grouped launch: 3 real GEMMs per bond,
// 2 * products * (2 chi)^2 * pad8(chi) each.
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
