// Two-site DMRG effective Hamiltonian matvec
//   out[a,s1,s2,b] = sum L[a,wl,a'] W[wl,wm,s1,t1] W[wm,wr,s2,t2] R[b,wr,b'] psi[a',t1,t2,b']
// evaluated right-to-left as three steps whose GEMMs are all "TN" (both
// operands K-major, read in place):
//   GEMM1  U[(a',t1,t2), (b,wr)]   = sum_b'       psi[(a',t1,t2), b'] R[(b,wr), b']
//          (stored transposed on the split path, U^T[(b,wr), (a',t1,t2)])
//   WW     V[(s1,s2,b), (wl,a')]   = sum_{wr,t1,t2} WW[wl,s1,s2,wr,t1,t2] U[(a',t1,t2),(b,wr)]
//   GEMM2  out[a, (s1,s2,b)]       = sum_{wl,a'}  L[a, (wl,a')] V[(s1,s2,b), (wl,a')]
// with WW[wl,s1,s2,wr,t1,t2] = sum_wm W[wl,wm,s1,t1] W[wm,wr,s2,t2] formed
// once per plan.  The W.W step writes V already transposed into GEMM2's
// K-major layout (and, on the split path, already split into bfloat16
// pieces), so no transpose is ever materialised for the GEMMs.
#include <cuda_bf16.h>

#include <string.h>

#include <algorithm>

#include "heff_plan.cuh"

namespace {

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ------------------------------------------------------------------ WW = W.W
// WW = sum_wm W1[wl,wm,s1,t1] W2[wm,wr,s2,t2]  (W1 on the left site, W2 on the right)
__global__ void k_ww_precompute(const double* __restrict__ W, const double* __restrict__ W2, int Dw, int d,
                                double* __restrict__ WW) {
  // WW index ((((wl*d + s1)*d + s2)*Dw + wr)*d + t1)*d + t2
  const int n = Dw * d * d * Dw * d * d;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int r = i;
    const int t2 = r % d; r /= d;
    const int t1 = r % d; r /= d;
    const int wr = r % Dw; r /= Dw;
    const int s2 = r % d; r /= d;
    const int s1 = r % d; r /= d;
    const int wl = r;
    double acc = 0.0;
    for (int wm = 0; wm < Dw; ++wm)
      acc += W[((wl * Dw + wm) * d + s1) * d + t1] * W2[((wm * Dw + wr) * d + s2) * d + t2];
    WW[i] = acc;
  }
}

// ------------------------------------------------------------------ W.W application
template <typename T>
struct WWArgs {
  T ww[HEFF_DW * 4 * HEFF_DW * 4];   // [wl][s][wr][t], s = (s1 s2), t = (t1 t2)
};

// FP64 path.  U [(a',t), (b,wr)].  One block: a' in [a0, a0+ATILE), b in
// [b0, b0+BT), one (a', b) pair per thread (ATILE*BT = 256).  The U rows
// (a', t) of the tile are staged in shared memory (row segments of BT*Dw
// contiguous values), then each thread forms the 20 outputs of its pair and
// writes them with a' fastest, which is contiguous along GEMM2's K dimension.
template <int ATILE, int BT>
__global__ void __launch_bounds__(ATILE * BT, 4) k_ww_apply(const WWArgs<double> args, const double* __restrict__ U,
                                                          int64_t chiL, int64_t chiR, double* __restrict__ V,
                                                          int64_t ldv) {
  constexpr int Dw = HEFF_DW, D2 = 4;
  constexpr int ROW = D2 * BT * Dw;   // staged values per a'
  __shared__ double Us[ATILE][ROW + 1];
  const int64_t a0 = (int64_t)blockIdx.y * ATILE;
  const int64_t b0 = (int64_t)blockIdx.x * BT;
  const int64_t ldu = chiR * Dw;
  for (int idx = threadIdx.x; idx < ATILE * D2 * BT * Dw; idx += ATILE * BT) {
    const int col = idx % (BT * Dw);
    const int rt = idx / (BT * Dw);   // a'_local * D2 + t
    const int al = rt / D2, t = rt % D2;
    const int64_t ap = a0 + al;
    const int64_t gcol = b0 * Dw + col;
    double v = 0.0;
    if (ap < chiL && gcol < ldu) v = U[(ap * D2 + t) * ldu + gcol];
    Us[al][t * BT * Dw + col] = v;
  }
  __syncthreads();
  const int al = threadIdx.x % ATILE, bl = threadIdx.x / ATILE;
  const int64_t ap = a0 + al, b = b0 + bl;
  if (ap >= chiL || b >= chiR) return;
  double in[D2 * Dw];
#pragma unroll
  for (int t = 0; t < D2; ++t)
#pragma unroll
    for (int wr = 0; wr < Dw; ++wr) in[t * Dw + wr] = Us[al][(t * BT + bl) * Dw + wr];
  const int64_t rowstep = chiR * ldv;   // s -> s + 1
  const int64_t base = b * ldv + ap;
#pragma unroll
  for (int s = 0; s < D2; ++s) {
#pragma unroll
    for (int wl = 0; wl < Dw; ++wl) {
      double acc = 0.0;
#pragma unroll
      for (int wr = 0; wr < Dw; ++wr)
#pragma unroll
        for (int t = 0; t < D2; ++t) acc += args.ww[((wl * D2 + s) * Dw + wr) * D2 + t] * in[t * Dw + wr];
      V[base + s * rowstep + wl * chiL] = acc;
    }
  }
}

// FP64 path for small bond dimensions: one thread per output (a', b, s, wl)
// instead of per pair, so a chi = 64 bond spreads over ~80k threads rather
// than 4k.  A block covers 8 a' x 2 b: their 8 x 4 x 2 x 5 = 320 inputs are
// staged in shared memory (one per thread) with the 400 W.W coefficients;
// a' runs fastest, so stores of one (s, wl) are contiguous along GEMM2's K.
constexpr int kWWsA = 8, kWWsB = 2, kWWsT = kWWsA * kWWsB * 20;   // 320 threads
__global__ void __launch_bounds__(kWWsT) k_ww_apply_small(const WWArgs<double> args, const double* __restrict__ U,
                                                          int64_t chiL, int64_t chiR, double* __restrict__ V,
                                                          int64_t ldv) {
  constexpr int Dw = HEFF_DW, D2 = 4;
  __shared__ double Us[kWWsA][D2][kWWsB][Dw];
  __shared__ double ww[Dw * D2 * Dw * D2];
  const int64_t a0 = (int64_t)blockIdx.y * kWWsA, b0 = (int64_t)blockIdx.x * kWWsB;
  const int64_t ldu = chiR * Dw;
  for (int i = threadIdx.x; i < Dw * D2 * Dw * D2; i += kWWsT) ww[i] = args.ww[i];
  {
    // staging: thread -> (wr, b, t, a') with wr fastest (contiguous (b, wr) runs of U rows)
    const int wr = threadIdx.x % Dw, bl = (threadIdx.x / Dw) % kWWsB, t = (threadIdx.x / (Dw * kWWsB)) % D2,
              al = threadIdx.x / (Dw * kWWsB * D2);
    const int64_t ap = a0 + al, b = b0 + bl;
    Us[al][t][bl][wr] = (ap < chiL && b < chiR) ? U[(ap * D2 + t) * ldu + b * Dw + wr] : 0.0;
  }
  __syncthreads();
  const int al = threadIdx.x % kWWsA, o = (threadIdx.x / kWWsA) % 20, bl = threadIdx.x / (kWWsA * 20);
  const int64_t ap = a0 + al, b = b0 + bl;
  if (ap >= chiL || b >= chiR) return;
  const int s = o % D2, wl = o / D2;
  double acc = 0.0;
#pragma unroll
  for (int wr = 0; wr < Dw; ++wr)
#pragma unroll
    for (int t = 0; t < D2; ++t) acc += ww[((wl * D2 + s) * Dw + wr) * D2 + t] * Us[al][t][bl][wr];
  V[b * ldv + ap + s * (chiR * ldv) + wl * chiL] = acc;
}

// Split path.  GEMM1 stores U transposed, U^T [(b,wr), (a',t)] (row length
// 4 chiL), so that one thread reads the NA*4 values (a', t), a' in
// [a0, a0+NA), of each of its five rows (b, wr) as contiguous float4s and a
// warp reads 32*NA*16 contiguous bytes per row, with no shared-memory
// staging.  The thread forms the 20 outputs (s, wl) of its NA pairs (a', b),
// splits them into bfloat16 pieces and stores NA consecutive a' per piece
// plane with one vector store (a' is GEMM2's K dimension).  Lanes run along
// a', so each warp store covers 32*NA*2 contiguous bytes.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// Only a' in [a_begin, a_end) is processed (a row range of psi).
template <int NA>
__global__ void __launch_bounds__(256) k_ww_split(const WWArgs<float> args, const float* __restrict__ Ut, int64_t chiL,
                                                  int64_t chiR, __nv_bfloat16* __restrict__ V, int64_t ldv,
                                                  int64_t plane, int64_t a_begin, int64_t a_end) {
  constexpr int Dw = HEFF_DW, D2 = 4;
  static_assert(NA == 2 || NA == 4, "NA");
  const int64_t nq = (a_end - a_begin + NA - 1) / NA;
  const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t q = idx % nq, b = idx / nq;
  if (b >= chiR) return;
  const int64_t a0 = a_begin + q * NA;
  const bool full = a0 + NA <= a_end;
  const int64_t ldu = 4 * chiL;
  float in[Dw][NA * D2];   // [wr][(a'-a0)*4 + t]
#pragma unroll
  for (int wr = 0; wr < Dw; ++wr) {
    const float* row = Ut + (b * Dw + wr) * ldu + a0 * D2;
    if (full) {
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const float4 v = __ldg((const float4*)row + j);
        in[wr][4 * j] = v.x;
        in[wr][4 * j + 1] = v.y;
        in[wr][4 * j + 2] = v.z;
        in[wr][4 * j + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NA * D2; ++j) in[wr][j] = a0 + j / D2 < a_end ? row[j] : 0.f;
    }
  }
  const bool vec = full && (chiL % NA == 0) && (a_begin % NA == 0);
#pragma unroll
  for (int s = 0; s < D2; ++s) {
#pragma unroll
    for (int wl = 0; wl < Dw; ++wl) {
      float acc[NA];
#pragma unroll
      for (int j = 0; j < NA; ++j) acc[j] = 0.f;
#pragma unroll
      for (int wr = 0; wr < Dw; ++wr)
#pragma unroll
        for (int t = 0; t < D2; ++t) {
          const float w = args.ww[((wl * D2 + s) * Dw + wr) * D2 + t];
#pragma unroll
          for (int j = 0; j < NA; ++j) acc[j] = fmaf(w, in[wr][j * D2 + t], acc[j]);
        }
      __nv_bfloat16 h[NA], m[NA], l[NA];
#pragma unroll
      for (int j = 0; j < NA; ++j) split3(acc[j], h[j], m[j], l[j]);
      const int64_t off = (s * chiR + b) * ldv + wl * chiL + a0;
      if (vec) {
        if constexpr (NA == 4) {
          uint2 ph, pm, pl;
          ph.x = pack_bf16x2(h[0], h[1]);
          ph.y = pack_bf16x2(h[2], h[3]);
          pm.x = pack_bf16x2(m[0], m[1]);
          pm.y = pack_bf16x2(m[2], m[3]);
          pl.x = pack_bf16x2(l[0], l[1]);
          pl.y = pack_bf16x2(l[2], l[3]);
          *(uint2*)(V + off) = ph;
          *(uint2*)(V + plane + off) = pm;
          *(uint2*)(V + 2 * plane + off) = pl;
        } else {
          *(uint32_t*)(V + off) = pack_bf16x2(h[0], h[1]);
          *(uint32_t*)(V + plane + off) = pack_bf16x2(m[0], m[1]);
          *(uint32_t*)(V + 2 * plane + off) = pack_bf16x2(l[0], l[1]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < NA; ++j)
          if (a0 + j < a_end) {
            V[off + j] = h[j];
            V[plane + off + j] = m[j];
            V[2 * plane + off + j] = l[j];
          }
      }
    }
  }
}

// The W.W step is FP64-pipe work (400 FMAs per (a', b) pair), so the tile
// shrinks for small bonds until the grid covers the SMs.
tci_status launch_ww_f64(tci_context ctx, const WWArgs<double>& args, const double* U, int64_t chiL, int64_t chiR,
                         double* V, int64_t ldv) {
  const int64_t sms = ctx->num_sms;
  auto blocks = [&](int at, int bt) { return ((chiR + bt - 1) / bt) * ((chiL + at - 1) / at); };
  if (blocks(16, 16) >= 2 * sms) {
    dim3 grid((unsigned)((chiR + 15) / 16), (unsigned)((chiL + 15) / 16));
    if (grid.y > 65535u) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "W.W step: chiL too large");
    k_ww_apply<16, 16><<<grid, 256, 0, ctx->stream>>>(args, U, chiL, chiR, V, ldv);
  } else if (blocks(8, 8) >= sms) {
    dim3 grid((unsigned)((chiR + 7) / 8), (unsigned)((chiL + 7) / 8));
    k_ww_apply<8, 8><<<grid, 64, 0, ctx->stream>>>(args, U, chiL, chiR, V, ldv);
  } else {   // few pairs: a thread per output
    dim3 grid((unsigned)((chiR + kWWsB - 1) / kWWsB), (unsigned)((chiL + kWWsA - 1) / kWWsA));
    if (grid.y > 65535u) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "W.W step: chiL too large");
    k_ww_apply_small<<<grid, kWWsT, 0, ctx->stream>>>(args, U, chiL, chiR, V, ldv);
  }
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

// na: a' per thread (2 or 4; 4 halves the store instructions, 2 doubles the
// resident warps), chosen by the autotuner.
tci_status launch_ww_split(tci_context ctx, const WWArgs<float>& args, const float* Ut, int64_t chiL, int64_t chiR,
                           void* V, int64_t ldv, int64_t plane, int na, int64_t a_begin = 0, int64_t a_end = -1) {
  if (a_end < 0) a_end = chiL;
  if (a_begin < 0 || a_end > chiL || a_begin >= a_end) return TCI_OK;
  const int64_t threads = (a_end - a_begin + na - 1) / na * chiR;
  const int64_t blocks = (threads + 255) / 256;
  if (blocks > 0x7fffffff) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "W.W step: too large");
  if (na == 2)
    k_ww_split<2><<<(unsigned)blocks, 256, 0, ctx->stream>>>(args, Ut, chiL, chiR, (__nv_bfloat16*)V, ldv, plane,
                                                             a_begin, a_end);
  else
    k_ww_split<4><<<(unsigned)blocks, 256, 0, ctx->stream>>>(args, Ut, chiL, chiR, (__nv_bfloat16*)V, ldv, plane,
                                                             a_begin, a_end);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

}  // namespace

// Time both W.W variants on the plan's current U (5 launches each) and keep
// the faster one in p->ww_na.
tci_status tci_heff_tune_ww(tci_heff_plan p, float* ms_out) {
  tci_context ctx = p->ctx;
  if (p->prec == TCI_PREC_NATIVE) return TCI_OK;
  WWArgs<float> args;
  for (int i = 0; i < HEFF_NWW; ++i) args.ww[i] = (float)p->ww[i];
  cudaEvent_t e0, e1;
  TCI_CUDA(ctx, cudaEventCreate(&e0));
  TCI_CUDA(ctx, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_na = p->ww_na;
  tci_status s = TCI_OK;
  const int cands[2] = {4, 2};
  for (int na : cands) {
    s = launch_ww_split(ctx, args, (const float*)p->U, p->chiL, p->chiR, p->Vp, p->Kp2, 4 * p->chiR * p->Kp2, na);
    if (s != TCI_OK) break;
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 5 && s == TCI_OK; ++r)
      s = launch_ww_split(ctx, args, (const float*)p->U, p->chiL, p->chiR, p->Vp, p->Kp2, 4 * p->chiR * p->Kp2, na);
    cudaEventRecord(e1, ctx->stream);
    if (s != TCI_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = tci_cuda_fail(ctx, e, "tune W.W");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_na = na;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == TCI_OK) {
    p->ww_na = best_na;
    if (ms_out) *ms_out = best / 5.f;
  }
  return s;
}

namespace {

int64_t pad8(int64_t x) { return (x + 7) / 8 * 8; }

}  // namespace

// ------------------------------------------------------------------ complex plans
// H_eff on C128 tensors through the library's own contraction (native
// complex FP64), in the order (psi R) W W L:
//   U0[x,i,j,b,r] = sum_y psi[x,i,j,y] R[b,r,y]
//   U1[x,i,b,m,u] = sum_{r,j} U0[x,i,j,b,r] W2[m,r,u,j]   (right site)
//   U2[x,b,u,s,w] = sum_{m,i} U1[x,i,b,m,u] W[w,m,s,i]    (left site)
//   out[a,s,u,b]  = sum_{w,x} L[a,w,x] U2[x,b,u,s,w]
static tci_status complex_plan_create(tci_context ctx, tci_tensor L, tci_tensor W, tci_tensor W2, tci_tensor R,
                                      tci_heff_plan* out) {
  if (L->dtype != TCI_C128 || W->dtype != TCI_C128 || W2->dtype != TCI_C128 || R->dtype != TCI_C128)
    return tci_fail(ctx, TCI_ERR_DTYPE, "heff_plan_create: a complex plan needs L, W, R all C128");
  if (L->order != 3 || R->order != 3 || W->order != 4)
    return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_create: L[chi,Dw,chi], W[Dw,Dw,d,d], R[chi,Dw,chi]");
  const int64_t Dw = W->shape[0], d = W->shape[2], chiL = L->shape[0], chiR = R->shape[0];
  if (Dw < 1 || d < 1 || W->shape[1] != Dw || W->shape[3] != d || L->shape[1] != Dw || L->shape[2] != chiL ||
      R->shape[1] != Dw || R->shape[2] != chiR || chiL < 1 || chiR < 1)
    return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_create: inconsistent complex L/W/R shapes");
  tci_heff_plan p = new tci_heff_plan_s();
  p->magic = kPlanMagic;
  p->ctx = ctx;
  p->chiL = chiL;
  p->chiR = chiR;
  p->prec = TCI_PREC_NATIVE;
  p->cplx = true;
  p->cd = d;
  p->cDw = Dw;
  tci_status s = tci_copy(ctx, L, &p->cL);
  if (s == TCI_OK) s = tci_copy(ctx, W, &p->cW);
  if (s == TCI_OK) s = tci_copy(ctx, W2, &p->cW2);
  if (s == TCI_OK) s = tci_copy(ctx, R, &p->cR);
  if (s != TCI_OK) {
    tci_heff_plan_destroy(&p);
    return s;
  }
  *out = p;
  return TCI_OK;
}

static tci_status complex_apply(tci_heff_plan p, tci_tensor psi, tci_tensor out) {
  tci_context ctx = p->ctx;
  for (tci_tensor t : {psi, out}) {
    if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "heff_apply: invalid tensor");
    if (t->dtype != TCI_C128) return tci_fail(ctx, TCI_ERR_DTYPE, "heff_apply: a complex plan takes C128 psi and out");
    if (t->order != 4 || t->shape[0] != p->chiL || t->shape[1] != p->cd || t->shape[2] != p->cd || t->shape[3] != p->chiR)
      return tci_fail(ctx, TCI_ERR_SHAPE, "heff_apply: psi and out must be [%lld,%lld,%lld,%lld]", (long long)p->chiL,
                      (long long)p->cd, (long long)p->cd, (long long)p->chiR);
  }
  if (psi->data == out->data) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "heff_apply: psi and out overlap");
  TCI_TRY(tci_contract(ctx, psi, "xijy", p->cR, "bry", &p->cU[0], "xijbr"));
  TCI_TRY(tci_contract(ctx, p->cU[0], "xijbr", p->cW2, "mruj", &p->cU[1], "xibmu"));
  TCI_TRY(tci_contract(ctx, p->cU[1], "xibmu", p->cW, "wmsi", &p->cU[2], "xbusw"));
  tci_tensor o = out;
  return tci_contract(ctx, p->cL, "awx", p->cU[2], "xbusw", &o, "asub");
}

// Matvec on raw device pointers of a complex plan (the Lanczos basis stores
// C128 vectors as interleaved FP64 pairs): borrowed C128 views kept in the
// plan, repointed at every call.
tci_status tci_heff_apply_complex_raw(tci_heff_plan p, const double* psi, double* out) {
  tci_context ctx = p->ctx;
  const int64_t shp[4] = {p->chiL, p->cd, p->cd, p->chiR};
  if (!p->cVin) TCI_TRY(tci_tensor_wrap(ctx, TCI_C128, 4, shp, nullptr, (void*)psi, &p->cVin));
  if (!p->cVout) TCI_TRY(tci_tensor_wrap(ctx, TCI_C128, 4, shp, nullptr, out, &p->cVout));
  p->cVin->data = (void*)psi;
  p->cVout->data = out;
  return complex_apply(p, p->cVin, p->cVout);
}

static tci_status complex_unsupported(tci_heff_plan p, const char* what) {
  return tci_fail(p->ctx, TCI_ERR_UNSUPPORTED, "%s: complex plans support tci_heff_apply only", what);
}

// ------------------------------------------------------------------ plan
extern "C" tci_status tci_heff_plan_create(tci_context ctx, tci_tensor L, tci_tensor W, tci_tensor R,
                                           tci_heff_plan* out) {
  return tci_heff_plan_create2(ctx, L, W, W, R, out);
}

extern "C" tci_status tci_heff_plan_create2(tci_context ctx, tci_tensor L, tci_tensor W, tci_tensor W2, tci_tensor R,
                                            tci_heff_plan* out) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "heff_plan_create");
  if (!out) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "heff_plan_create: NULL output");
  *out = nullptr;
  if (!tci_ten_ok(L) || !tci_ten_ok(W) || !tci_ten_ok(W2) || !tci_ten_ok(R))
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "heff_plan_create: invalid tensor");
  if (W2->dtype != W->dtype || W2->order != W->order || !tci_is_rowmajor(W2))
    return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_create: W2 must be a row-major tensor of W's dtype and shape");
  for (int i = 0; i < W->order; ++i)
    if (W2->shape[i] != W->shape[i]) return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_create: W2 must have W's shape");
  if (L->dtype == TCI_C128 || W->dtype == TCI_C128 || R->dtype == TCI_C128)
    return complex_plan_create(ctx, L, W, W2, R, out);
  if (L->dtype != TCI_F64 || W->dtype != TCI_F64 || R->dtype != TCI_F64)
    return tci_fail(ctx, TCI_ERR_DTYPE, "heff_plan_create: L, W, R must be F64");
  if (L->order != 3 || R->order != 3 || W->order != 4) return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_create: L[chi,Dw,chi], W[Dw,Dw,d,d], R[chi,Dw,chi]");
  const int64_t Dw = W->shape[0], d = W->shape[2];
  if (Dw != HEFF_DW || W->shape[1] != Dw || d != 2 || W->shape[3] != d)
    return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "heff_plan_create: this build supports Dw = %d, d = 2", HEFF_DW);
  const int64_t chiL = L->shape[0], chiR = R->shape[0];
  if (L->shape[1] != Dw || L->shape[2] != chiL || R->shape[1] != Dw || R->shape[2] != chiR || chiL <= 0 || chiR <= 0)
    return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_create: inconsistent L/R shapes");
  if (!tci_is_rowmajor(L) || !tci_is_rowmajor(W) || !tci_is_rowmajor(R))
    return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_create: L, W, R must be row-major contiguous");
  vs.info = "chiL=" + std::to_string(chiL) + " chiR=" + std::to_string(chiR);

  tci_heff_plan p = new tci_heff_plan_s();
  p->magic = kPlanMagic;
  p->ctx = ctx;
  p->chiL = chiL;
  p->chiR = chiR;
  p->prec = ctx->precision;
  p->products = ctx->precision == TCI_PREC_SPLIT_BF16_3 ? 3 : 6;
  p->chunk_k = ctx->split_chunk_k;
  p->xchunk_k = ctx->split_xchunk_k;
  const int64_t n_psi = chiL * 4 * chiR;
  const int64_t nU = chiL * 4 * chiR * Dw;
  auto fail = [&](tci_status s) {
    tci_heff_plan pp = p;
    tci_heff_plan_destroy(&pp);
    return s;
  };
  tci_status s;
  // WW (FP64) on the device, then a host copy for the kernel arguments
  double* dWW = nullptr;
  if ((s = tci_dev_alloc(ctx, sizeof(double) * HEFF_NWW, (void**)&dWW)) != TCI_OK) return fail(s);
  k_ww_precompute<<<1, 256, 0, ctx->stream>>>((const double*)W->data, (const double*)W2->data, (int)Dw, (int)d, dWW);
  cudaError_t e = cudaMemcpyAsync(p->ww, dWW, sizeof(double) * HEFF_NWW, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  tci_dev_free(dWW);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "heff_plan_create: WW"));

  const size_t ubytes = (p->prec == TCI_PREC_NATIVE ? sizeof(double) : sizeof(float)) * nU;
  if ((s = tci_dev_alloc(ctx, ubytes, (void**)&p->U)) != TCI_OK) return fail(s);
  if (p->prec == TCI_PREC_NATIVE) {
    if ((s = tci_dev_alloc(ctx, sizeof(double) * chiL * Dw * chiL, (void**)&p->L64)) != TCI_OK) return fail(s);
    if ((s = tci_dev_alloc(ctx, sizeof(double) * chiR * Dw * chiR, (void**)&p->R64)) != TCI_OK) return fail(s);
    if ((s = tci_dev_alloc(ctx, sizeof(double) * nU, (void**)&p->V64)) != TCI_OK) return fail(s);
    e = cudaMemcpyAsync(p->L64, L->data, sizeof(double) * chiL * Dw * chiL, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->R64, R->data, sizeof(double) * chiR * Dw * chiR, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "heff_plan_create: copy L/R"));
    // split-K partials of the two GEMMs, owned by the plan (no allocation per matvec)
    p->ws_bytes = std::max(tci_gemm_native_workspace(ctx, TCI_F64, 1, chiL * 4, chiR * Dw, chiR),
                           tci_gemm_native_workspace(ctx, TCI_F64, 1, chiL, 4 * chiR, Dw * chiL));
    if (p->ws_bytes && (s = tci_dev_alloc(ctx, p->ws_bytes, &p->ws)) != TCI_OK) return fail(s);
  } else {
    p->Kp1 = pad8(chiR);
    p->Kp2 = pad8(Dw * chiL);
    if ((s = tci_dev_alloc(ctx, 2 * 3 * chiL * p->Kp2, (void**)&p->Lp)) != TCI_OK) return fail(s);
    if ((s = tci_dev_alloc(ctx, 2 * 3 * chiR * Dw * p->Kp1, (void**)&p->Rp)) != TCI_OK) return fail(s);
    if ((s = tci_dev_alloc(ctx, 2 * 3 * chiL * 4 * p->Kp1, (void**)&p->psip)) != TCI_OK) return fail(s);
    if ((s = tci_dev_alloc(ctx, 2 * 3 * 4 * chiR * p->Kp2, (void**)&p->Vp)) != TCI_OK) return fail(s);
    // padded K columns of V stay zero (the W.W step writes valid columns only)
    if (p->Kp2 != Dw * chiL) {
      e = cudaMemsetAsync(p->Vp, 0, 2 * 3 * 4 * chiR * p->Kp2, ctx->stream);
      if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "heff_plan_create: memset"));
    }
    // L as [a, (wl,a')] and R as [(b,wr), b'] : K-major rows of the GEMMs
    if ((s = tci_launch_split3(ctx, TCI_F64, L->data, chiL, Dw * chiL, Dw * chiL, 1, p->Lp, p->Kp2)) != TCI_OK) return fail(s);
    if ((s = tci_launch_split3(ctx, TCI_F64, R->data, chiR * Dw, chiR, chiR, 1, p->Rp, p->Kp1)) != TCI_OK) return fail(s);
  }
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "heff_plan_create"));
  (void)n_psi;
  *out = p;
  return TCI_OK;
}

// New environments (and MPO tensors) of the same shapes for an existing real
// plan: L and R copied (FP64 plan) or re-split (split plan) into the plan's
// own buffers, stream-ordered; W.W recomputed unless same_mpo.  A changed W.W
// drops the plan's Lanczos graph (its kernels take W.W by value).
tci_status tci_heff_plan_reload_impl(tci_heff_plan p, tci_tensor L, tci_tensor W, tci_tensor W2, tci_tensor R,
                                     bool same_mpo) {
  tci_context ctx = p->ctx;
  if (p->cplx) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "heff_plan_reload: real plans only");
  if (!W2) W2 = W;
  const int64_t Dw = HEFF_DW, chiL = p->chiL, chiR = p->chiR;
  for (tci_tensor t : {L, W, W2, R}) {
    if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "heff_plan_reload: invalid L, W, W2 or R");
    if (t->dtype != TCI_F64) return tci_fail(ctx, TCI_ERR_DTYPE, "heff_plan_reload: L, W, W2, R must be F64");
    if (!tci_is_rowmajor(t)) return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_reload: L, W, W2, R must be row-major");
  }
  if (L->order != 3 || R->order != 3 || W->order != 4 || W2->order != 4 || L->shape[0] != chiL || L->shape[1] != Dw ||
      L->shape[2] != chiL || R->shape[0] != chiR || R->shape[1] != Dw || R->shape[2] != chiR || W->shape[0] != Dw ||
      W->shape[1] != Dw || W->shape[2] != 2 || W->shape[3] != 2)
    return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_reload: shapes differ from the plan's");
  for (int i = 0; i < 4; ++i)
    if (W2->shape[i] != W->shape[i]) return tci_fail(ctx, TCI_ERR_SHAPE, "heff_plan_reload: W2 must have W's shape");
  if (!same_mpo) {
    double* dWW = nullptr;
    TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * HEFF_NWW, (void**)&dWW));
    k_ww_precompute<<<1, 256, 0, ctx->stream>>>((const double*)W->data, (const double*)W2->data, (int)Dw, 2, dWW);
    double ww[HEFF_NWW];
    cudaError_t e = cudaMemcpyAsync(ww, dWW, sizeof(ww), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    tci_dev_free(dWW);
    if (e != cudaSuccess) return tci_cuda_fail(ctx, e, "heff_plan_reload: WW");
    if (memcmp(ww, p->ww, sizeof(ww)) != 0) {
      memcpy(p->ww, ww, sizeof(ww));
      tci_graph_destroy(&p->lz_graph);
      p->lz_graph_key.clear();
      p->lz_last_key.clear();
    }
  }
  if (p->prec == TCI_PREC_NATIVE) {
    TCI_CUDA(ctx, cudaMemcpyAsync(p->L64, L->data, sizeof(double) * chiL * Dw * chiL, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    TCI_CUDA(ctx, cudaMemcpyAsync(p->R64, R->data, sizeof(double) * chiR * Dw * chiR, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  } else {
    TCI_TRY(tci_launch_split3(ctx, TCI_F64, L->data, chiL, Dw * chiL, Dw * chiL, 1, p->Lp, p->Kp2));
    TCI_TRY(tci_launch_split3(ctx, TCI_F64, R->data, chiR * Dw, chiR, chiR, 1, p->Rp, p->Kp1));
  }
  return TCI_OK;
}

extern "C" tci_status tci_heff_plan_reload(tci_heff_plan p, tci_tensor L, tci_tensor W, tci_tensor W2, tci_tensor R) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_plan_reload: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  TciVerboseScope vs(p->ctx, "heff_plan_reload");
  return tci_heff_plan_reload_impl(p, L, W, W2, R, false);
}

extern "C" tci_status tci_heff_plan_destroy(tci_heff_plan* pp) {
  if (!pp || !*pp || (*pp)->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_plan_destroy: invalid plan");
  tci_heff_plan p = *pp;
  if (tci_ctx_ok(p->ctx)) cudaStreamSynchronize(p->ctx->stream);
  void* bufs[] = {p->U, p->L64, p->R64, p->V64, p->Lp, p->Rp, p->psip, p->Vp, p->d_stage_in, p->d_stage_out,
                  p->lz_V, p->lz_Vs, p->lz_w, p->lz_scal, p->lz_part, p->lz_x64, p->lz_o64, p->ws};
  for (void* b : bufs) tci_dev_free(b);
  for (tci_tensor* t : {&p->cL, &p->cW, &p->cW2, &p->cR, &p->cU[0], &p->cU[1], &p->cU[2], &p->cVin, &p->cVout})
    if (*t) tci_tensor_free(t);
  for (int i = 0; i < 8; ++i) {
    if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
    if (p->ev_out[i]) cudaEventDestroy(p->ev_out[i]);
  }
  if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
  if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
  tci_graph_destroy(&p->lz_graph);
  p->magic = 0;
  delete p;
  *pp = nullptr;
  return TCI_OK;
}

extern "C" double tci_heff_flops(tci_heff_plan p) {
  if (!p || p->magic != kPlanMagic) return 0.0;
  if (p->cplx) {   // complex multiply-adds of the four contractions, 8 real flops each
    const double chiL = (double)p->chiL, chiR = (double)p->chiR, d = (double)p->cd, Dw = (double)p->cDw;
    return 8.0 * (chiL * d * d * chiR * Dw * (chiL + chiR) + 2.0 * chiL * chiR * d * d * d * Dw * Dw);
  }
  const double chiL = (double)p->chiL, chiR = (double)p->chiR, d = 2.0, Dw = HEFF_DW;
  return 2.0 * chiL * d * d * chiR * Dw * (chiL + chiR) + 2.0 * chiL * chiR * d * d * d * d * Dw * Dw;
}

// ------------------------------------------------------------------ apply
static tci_status check_vec(tci_heff_plan p, tci_tensor t, const char* what);
tci_status tci_heff_apply_raw(tci_heff_plan p, const double* psi, void* out, bool psi_presplit, int out_mode) {
  tci_context ctx = p->ctx;
  const int64_t chiL = p->chiL, chiR = p->chiR, Dw = HEFF_DW;
  if (p->prec == TCI_PREC_NATIVE) {
    if (out_mode != 0 || psi_presplit) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "heff_apply: FP64 plan writes FP64");
    WWArgs<double> args;
    for (int i = 0; i < HEFF_NWW; ++i) args.ww[i] = p->ww[i];
    TCI_TRY(tci_gemm_native_batched_ws(ctx, TCI_F64, 1, chiL * 4, chiR * Dw, chiR, psi, 0, chiR, 1, p->R64, 0, chiR, 1,
                                       p->U, 0, chiR * Dw, 1, p->ws, p->ws_bytes));
    TCI_TRY(launch_ww_f64(ctx, args, (const double*)p->U, chiL, chiR, p->V64, Dw * chiL));
    TCI_TRY(tci_gemm_native_batched_ws(ctx, TCI_F64, 1, chiL, 4 * chiR, Dw * chiL, p->L64, 0, Dw * chiL, 1, p->V64, 0,
                                       Dw * chiL, 1, out, 0, 4 * chiR, 1, p->ws, p->ws_bytes));
    return TCI_OK;
  }
  WWArgs<float> args;
  for (int i = 0; i < HEFF_NWW; ++i) args.ww[i] = (float)p->ww[i];
  if (!psi_presplit) TCI_TRY(tci_launch_split3(ctx, TCI_F64, psi, chiL * 4, chiR, chiR, 1, p->psip, p->Kp1));
  // GEMM1 stores U transposed: U^T[(b,wr), (a',t)] (m stride 1, n stride 4 chiL)
  TCI_TRY(tci_gemm_split_bf16(ctx, chiL * 4, chiR * Dw, p->Kp1, p->psip, p->Rp, p->U, 1, 1, chiL * 4, p->products,
                              p->chunk_k, p->xchunk_k, p->raster));
  TCI_TRY(launch_ww_split(ctx, args, (const float*)p->U, chiL, chiR, p->Vp, p->Kp2, 4 * chiR * p->Kp2, p->ww_na));
  TCI_TRY(tci_gemm_split_bf16(ctx, chiL, 4 * chiR, p->Kp2, p->Lp, p->Vp, out, out_mode, 4 * chiR, 1, p->products,
                              p->chunk_k, p->xchunk_k, p->raster));
  return TCI_OK;
}

// Split plan, psi already split into p->psip, FP64 output: the matvec with
// the dot products of its output folded into GEMM2 (see
// tci_gemm_split_bf16_dots): part rows 0..nv-1 receive the partial sums of
// <V_i, out>, row nv those of <out, out>, over *grid CTAs.
tci_status tci_heff_apply_raw_dots(tci_heff_plan p, double* out, const double* V, int64_t ldv, int nv, double* part,
                                   int part_stride, int* grid) {
  tci_context ctx = p->ctx;
  if (p->prec == TCI_PREC_NATIVE || p->cplx) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "heff_apply_dots: split plans only");
  const int64_t chiL = p->chiL, chiR = p->chiR, Dw = HEFF_DW;
  WWArgs<float> args;
  for (int i = 0; i < HEFF_NWW; ++i) args.ww[i] = (float)p->ww[i];
  TCI_TRY(tci_gemm_split_bf16(ctx, chiL * 4, chiR * Dw, p->Kp1, p->psip, p->Rp, p->U, 1, 1, chiL * 4, p->products,
                              p->chunk_k, p->xchunk_k, p->raster));
  TCI_TRY(launch_ww_split(ctx, args, (const float*)p->U, chiL, chiR, p->Vp, p->Kp2, 4 * chiR * p->Kp2, p->ww_na));
  return tci_gemm_split_bf16_dots(ctx, chiL, 4 * chiR, p->Kp2, p->Lp, p->Vp, out, p->products, p->chunk_k,
                                  p->xchunk_k, p->raster, V, ldv, nv, part, part_stride, grid);
}

// Same as tci_heff_apply_raw with CUDA events between the stages (split,
// GEMM1, W.W, GEMM2); ms[0..3] receive the stage durations.
static tci_status apply_timed(tci_heff_plan p, const double* psi, double* out, float* ms) {
  tci_context ctx = p->ctx;
  const int64_t chiL = p->chiL, chiR = p->chiR, Dw = HEFF_DW;
  cudaEvent_t ev[5];
  for (auto& e : ev) TCI_CUDA(ctx, cudaEventCreate(&e));
  tci_status s = TCI_OK;
  TCI_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream));
  if (p->prec == TCI_PREC_NATIVE) {
    WWArgs<double> args;
    for (int i = 0; i < HEFF_NWW; ++i) args.ww[i] = p->ww[i];
    TCI_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
    if (s == TCI_OK) s = tci_gemm_native(ctx, TCI_F64, chiL * 4, chiR * Dw, chiR, psi, chiR, 1, p->R64, chiR, 1, p->U, chiR * Dw, 1);
    TCI_CUDA(ctx, cudaEventRecord(ev[2], ctx->stream));
    if (s == TCI_OK) s = launch_ww_f64(ctx, args, (const double*)p->U, chiL, chiR, p->V64, Dw * chiL);
    TCI_CUDA(ctx, cudaEventRecord(ev[3], ctx->stream));
    if (s == TCI_OK) s = tci_gemm_native(ctx, TCI_F64, chiL, 4 * chiR, Dw * chiL, p->L64, Dw * chiL, 1, p->V64, Dw * chiL, 1, out, 4 * chiR, 1);
  } else {
    WWArgs<float> args;
    for (int i = 0; i < HEFF_NWW; ++i) args.ww[i] = (float)p->ww[i];
    s = tci_launch_split3(ctx, TCI_F64, psi, chiL * 4, chiR, chiR, 1, p->psip, p->Kp1);
    TCI_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
    if (s == TCI_OK) s = tci_gemm_split_bf16(ctx, chiL * 4, chiR * Dw, p->Kp1, p->psip, p->Rp, p->U, 1, 1, chiL * 4, p->products, p->chunk_k, p->xchunk_k, p->raster);
    TCI_CUDA(ctx, cudaEventRecord(ev[2], ctx->stream));
    if (s == TCI_OK) s = launch_ww_split(ctx, args, (const float*)p->U, chiL, chiR, p->Vp, p->Kp2, 4 * chiR * p->Kp2, p->ww_na);
    TCI_CUDA(ctx, cudaEventRecord(ev[3], ctx->stream));
    if (s == TCI_OK) s = tci_gemm_split_bf16(ctx, chiL, 4 * chiR, p->Kp2, p->Lp, p->Vp, out, 0, 4 * chiR, 1, p->products, p->chunk_k, p->xchunk_k, p->raster);
  }
  TCI_CUDA(ctx, cudaEventRecord(ev[4], ctx->stream));
  TCI_CUDA(ctx, cudaEventSynchronize(ev[4]));
  for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  for (auto& e : ev) cudaEventDestroy(e);
  return s;
}

extern "C" tci_status tci_heff_apply_timed(tci_heff_plan p, tci_tensor psi, tci_tensor out, float* stage_ms) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_apply_timed: invalid plan");
  if (p->cplx) return complex_unsupported(p, "heff_apply_timed");
  TCI_CHECK_CTX(p->ctx);
  if (!stage_ms) return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "heff_apply_timed: NULL stage_ms");
  TCI_TRY(check_vec(p, psi, "heff_apply_timed psi"));
  TCI_TRY(check_vec(p, out, "heff_apply_timed out"));
  return apply_timed(p, (const double*)psi->data, (double*)out->data, stage_ms);
}

static tci_status check_vec(tci_heff_plan p, tci_tensor t, const char* what) {
  tci_context ctx = p->ctx;
  if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "%s: invalid tensor", what);
  if (t->dtype != TCI_F64) return tci_fail(ctx, TCI_ERR_DTYPE, "%s: must be F64", what);
  if (t->order != 4 || t->shape[0] != p->chiL || t->shape[1] != 2 || t->shape[2] != 2 || t->shape[3] != p->chiR)
    return tci_fail(ctx, TCI_ERR_SHAPE, "%s: expected [%lld,2,2,%lld]", what, (long long)p->chiL, (long long)p->chiR);
  if (!tci_is_rowmajor(t)) return tci_fail(ctx, TCI_ERR_SHAPE, "%s: must be row-major contiguous", what);
  return TCI_OK;
}

extern "C" tci_status tci_heff_apply(tci_heff_plan p, tci_tensor psi, tci_tensor out) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_apply: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  TciVerboseScope vs(p->ctx, "heff_apply");
  if (p->cplx) return complex_apply(p, psi, out);
  TCI_TRY(check_vec(p, psi, "heff_apply psi"));
  TCI_TRY(check_vec(p, out, "heff_apply out"));
  if (psi->data == out->data) return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "heff_apply: psi and out overlap");
  return tci_heff_apply_raw(p, (const double*)psi->data, (double*)out->data, false);
}

// Host-buffer matvec on a split-BF16 plan with the copies overlapped: psi
// is copied in chunks of a' rows on one copy stream while the compute stream
// splits each arrived chunk, runs GEMM1 on its rows and W.W on its a' range;
// GEMM2 then runs in chunks of output rows a, each copied back on a second
// copy stream as soon as it is done.
static tci_status apply_host_pipelined(tci_heff_plan p, const double* psi_host, double* out_host) {
  tci_context ctx = p->ctx;
  const int64_t chiL = p->chiL, chiR = p->chiR, Dw = HEFF_DW;
  if (!p->s_h2d) {
    TCI_CUDA(ctx, cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking));
    TCI_CUDA(ctx, cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking));
    for (int i = 0; i < 8; ++i) {
      TCI_CUDA(ctx, cudaEventCreateWithFlags(&p->ev_in[i], cudaEventDisableTiming));
      TCI_CUDA(ctx, cudaEventCreateWithFlags(&p->ev_out[i], cudaEventDisableTiming));
    }
  }
  const int nch = chiL >= 256 ? 4 : 1;
  int64_t bnd[5];
  for (int c = 0; c <= nch; ++c) bnd[c] = c == nch ? chiL : (c * chiL / nch) / 8 * 8;
  WWArgs<float> args;
  for (int i = 0; i < HEFF_NWW; ++i) args.ww[i] = (float)p->ww[i];
  // the copy stream starts after the compute stream's earlier work (staging buffers are stream-ordered)
  TCI_CUDA(ctx, cudaEventRecord(p->ev_in[7], ctx->stream));
  TCI_CUDA(ctx, cudaStreamWaitEvent(p->s_h2d, p->ev_in[7], 0));
  // psi rows (a', t1, t2) of a' in [a0, a1) in, as they arrive
  for (int c = 0; c < nch; ++c) {
    const int64_t r0 = 4 * bnd[c] * chiR, n = 4 * (bnd[c + 1] - bnd[c]) * chiR;
    if (n == 0) continue;
    TCI_CUDA(ctx, cudaMemcpyAsync(p->d_stage_in + r0, psi_host + r0, n * sizeof(double), cudaMemcpyHostToDevice,
                                  p->s_h2d));
    TCI_CUDA(ctx, cudaEventRecord(p->ev_in[c], p->s_h2d));
  }
  __nv_bfloat16* psip = (__nv_bfloat16*)p->psip;
  for (int c = 0; c < nch; ++c) {
    const int64_t a0 = bnd[c], a1 = bnd[c + 1];
    if (a1 == a0) continue;
    TCI_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, p->ev_in[c], 0));
    TCI_TRY(tci_launch_split3(ctx, TCI_F64, p->d_stage_in + 4 * a0 * chiR, 4 * (a1 - a0), chiR, chiR, 1,
                              psip + 4 * a0 * p->Kp1, p->Kp1, 4 * chiL));
    TCI_TRY(tci_gemm_split_bf16_sub(ctx, 4 * (a1 - a0), chiR * Dw, p->Kp1, psip + 4 * a0 * p->Kp1, 4 * chiL, p->Rp,
                                    chiR * Dw, (float*)p->U + 4 * a0, 1, 1, chiL * 4, p->products, p->chunk_k,
                                    p->xchunk_k, p->raster));
    TCI_TRY(launch_ww_split(ctx, args, (const float*)p->U, chiL, chiR, p->Vp, p->Kp2, 4 * chiR * p->Kp2, p->ww_na, a0,
                            a1));
  }
  // output rows a in [a0, a1) out, as they are done
  const __nv_bfloat16* Lp = (const __nv_bfloat16*)p->Lp;
  for (int c = 0; c < nch; ++c) {
    const int64_t a0 = bnd[c], a1 = bnd[c + 1];
    if (a1 == a0) continue;
    TCI_TRY(tci_gemm_split_bf16_sub(ctx, a1 - a0, 4 * chiR, p->Kp2, Lp + a0 * p->Kp2, chiL, p->Vp, 4 * chiR,
                                    p->d_stage_out + a0 * 4 * chiR, 0, 4 * chiR, 1, p->products, p->chunk_k,
                                    p->xchunk_k, p->raster));
    TCI_CUDA(ctx, cudaEventRecord(p->ev_out[c], ctx->stream));
    TCI_CUDA(ctx, cudaStreamWaitEvent(p->s_d2h, p->ev_out[c], 0));
    TCI_CUDA(ctx, cudaMemcpyAsync(out_host + a0 * 4 * chiR, p->d_stage_out + a0 * 4 * chiR,
                                  (a1 - a0) * 4 * chiR * sizeof(double), cudaMemcpyDeviceToHost, p->s_d2h));
  }
  TCI_CUDA(ctx, cudaStreamSynchronize(p->s_d2h));
  return tci_synchronize(ctx);
}

extern "C" tci_status tci_heff_apply_host(tci_heff_plan p, const double* psi_host, double* out_host) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_apply_host: invalid plan");
  if (p->cplx) return complex_unsupported(p, "heff_apply_host");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "heff_apply_host");
  if (!psi_host || !out_host) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "heff_apply_host: NULL buffer");
  const size_t bytes = sizeof(double) * p->chiL * 4 * p->chiR;
  if (!p->d_stage_in) {
    TCI_TRY(tci_dev_alloc(ctx, bytes, (void**)&p->d_stage_in));
    TCI_TRY(tci_dev_alloc(ctx, bytes, (void**)&p->d_stage_out));
  }
  if (p->prec != TCI_PREC_NATIVE) return apply_host_pipelined(p, psi_host, out_host);
  TCI_CUDA(ctx, cudaMemcpyAsync(p->d_stage_in, psi_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  TCI_TRY(tci_heff_apply_raw(p, p->d_stage_in, p->d_stage_out, false));
  TCI_CUDA(ctx, cudaMemcpyAsync(out_host, p->d_stage_out, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  return tci_synchronize(ctx);
}
