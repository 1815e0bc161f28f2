// U(1) block-sparse two-site H_eff (charge-conserving tensors; the paper
// names symmetric tensors as future TCI work in Sec. IV).  The result is the
// dense H_eff of the zero-filled tensors restricted to the allowed blocks;
// only charge-allowed block products are computed.
//
// Blocks and their canonical packed order (each block row-major, blocks
// concatenated without gaps):
//   psi/out (ia, t1, t2, ib)  q_ib = q_ia + c(t1) + c(t2)   for ia, t1, t2
//   L (ia, w, ja), R (ib, w, jb)   q_j = q_i + Delta(w)        for i, w
// where q are the sector charges, c the physical charges and Delta the MPO
// channel charges; sector indices follow the caller's sector order.
//
// Per matvec (all block GEMMs of a stage in ONE grouped persistent launch):
//   1. split psi blocks into bfloat16 pieces (K-major, padded to 8)
//   2. grouped GEMM1, one problem per sector ib': the psi blocks P = (ia',
//      t1, t2, ib') that share ib' are stacked along M (their pieces are
//      split straight into the stack), so one problem computes every
//        U_P[a', (wr, b)] = sum_b' psi_P[a', b'] Rg_ib'[(wr, b), b']
//      Rg_ib' stacks the R blocks (ib(wr), wr, ib') along rows (plan time)
//   3. W.W tasks, one per sector pair (ja, ib): V[(s1 s2, b), (wl, a')] from
//      the (t1 t2, wr) sub-blocks of the U_P that exist, written as pieces
//      straight into GEMM2's K-major operand
//   4. grouped GEMM2, one problem per sector ia: the output blocks O = (ia,
//      s1, s2, ib) that share ia (and so Lg_ia) are stacked along N, so one
//      problem computes every
//        out_O[a, b] = sum_{wl, a'} Lg_ia[a, (wl, a')] Vg_O[b, (wl, a')]
//      Lg_ia concatenates the L blocks (ia, wl, ja(wl)) along K (plan time);
//      the stacked result lands in a staging buffer and an unpack pass
//      writes the packed output blocks.
// Stacking fills the 128-row / 128- or 64-column tiles that single small
// sector blocks would leave mostly empty (the total chi = 2048, 31-sector
// workload: 558 -> 361 GEMM1 tiles, 200 -> 116 GEMM2 tiles).
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "tci_internal.cuh"

#define BS_DW 5
#define BS_D 2

constexpr int kBsMagic = 0xb5b5e001;

namespace {

int64_t pad8(int64_t x) { return (x + 7) / 8 * 8; }
// FP32 row stride of a GEMM output: a multiple of 4 elements keeps every row
// 16-byte aligned, so the epilogue stores rows as float4 vectors
int64_t pad4(int64_t x) { return (x + 3) / 4 * 4; }
int64_t al256(int64_t bytes) { return (bytes + 255) / 256 * 256; }

// split FP32 rows into bf16 piece planes [3][rows][Kp] (zero in k >= K)
struct SplitJob {
  int64_t src_off;   // element offset of the block in the packed FP32 source
  int64_t rows, K, ld_src, Kp;
  int64_t dst_off;   // bf16 element offset of plane 0 in the destination arena
  int64_t plane;     // elements between piece planes (the block may sit inside a stack)
};

// The per-call passes (psi split, output unpack) run over a plan-time table of
// chunks, each a run of one job's work items: the grid is as large as the work,
// instead of one grid row per job sized for the largest block (most of whose
// blocks would find nothing to do).  Offsets inside a job are 32-bit (the plan
// checks they fit).
struct BsChunk {
  int job;
  int start;   // first work item of the chunk inside its job
};
constexpr int kSplitOctets = 256;    // work items (8 consecutive k of one row) per split chunk
constexpr int kUnpackElems = 1024;   // elements per unpack chunk (4 per thread)

// One work item per thread: eight consecutive k of one row, written as one
// 16-byte vector per piece plane (Kp, the plane stride and the destination
// offset are multiples of 8 elements).
__global__ void __launch_bounds__(kSplitOctets) k_bs_split(const BsChunk* __restrict__ chunks,
                                                           const SplitJob* __restrict__ jobs,
                                                           const float* __restrict__ src,
                                                           __nv_bfloat16* __restrict__ dst) {
  const BsChunk c = chunks[blockIdx.x];
  const SplitJob j = jobs[c.job];
  const int oct = (int)(j.Kp / 8);
  const int item = c.start + threadIdx.x;
  if (item >= (int)j.rows * oct) return;
  const int r = item / oct, k0 = (item - r * oct) * 8, K = (int)j.K;
  const float* s = src + j.src_off + (int64_t)r * j.ld_src;
  __align__(16) __nv_bfloat16 h[8], m[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const float x = k0 + e < K ? s[k0 + e] : 0.f;
    h[e] = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h[e]);
    m[e] = __float2bfloat16_rn(r1);
    l[e] = __float2bfloat16_rn(r1 - __bfloat162float(m[e]));
  }
  __nv_bfloat16* d = dst + j.dst_off + (int64_t)r * j.Kp + k0;
  *reinterpret_cast<uint4*>(d) = *reinterpret_cast<const uint4*>(h);
  *reinterpret_cast<uint4*>(d + j.plane) = *reinterpret_cast<const uint4*>(m);
  *reinterpret_cast<uint4*>(d + 2 * j.plane) = *reinterpret_cast<const uint4*>(l);
}

// split a FP32 block [rows][K] (row stride ld_src) into the column slice
// [dst_off + r*dst_ld + k] of bf16 piece planes dst_plane elements apart
struct SliceJob {
  int64_t src_off, rows, K, ld_src, dst_off, dst_ld, dst_plane;
};

__global__ void k_bs_split_slice(const SliceJob* __restrict__ jobs, const float* __restrict__ src,
                                 __nv_bfloat16* __restrict__ dst) {
  const SliceJob j = jobs[blockIdx.y];
  const int64_t n = j.rows * j.K;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / j.K, k = i - r * j.K;
    const float x = src[j.src_off + r * j.ld_src + k];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
    const int64_t o = j.dst_off + r * j.dst_ld + k;
    dst[o] = h;
    dst[j.dst_plane + o] = m;
    dst[2 * j.dst_plane + o] = l;
  }
}

// stacked GEMM2 result -> packed output block: out[dst_off + r*cols + c] =
// stage[src_off + r*ld_src + c], or 0 where src_off < 0 (no GEMM writes it)
struct UnpackJob {
  int64_t src_off, ld_src, rows, cols, dst_off;
};

__global__ void __launch_bounds__(256) k_bs_unpack(const BsChunk* __restrict__ chunks,
                                                   const UnpackJob* __restrict__ jobs,
                                                   const float* __restrict__ stage, float* __restrict__ out) {
  const BsChunk c = chunks[blockIdx.x];
  const UnpackJob j = jobs[c.job];
  const int n = (int)(j.rows * j.cols), cols = (int)j.cols;
  const float* sp = stage + (j.src_off >= 0 ? j.src_off : 0);
  float* op = out + j.dst_off;
#pragma unroll
  for (int e = 0; e < kUnpackElems / 256; ++e) {
    const int i = c.start + e * 256 + threadIdx.x;
    if (i >= n) break;
    const int r = i / cols, cc = i - r * cols;
    op[i] = j.src_off >= 0 ? sp[(int64_t)r * j.ld_src + cc] : 0.f;
  }
}

template <typename Job>
tci_status run_jobs(tci_context ctx, const std::vector<Job>& jobs, int64_t max_work,
                    void (*kern)(const Job*, const float*, __nv_bfloat16*), const float* src, __nv_bfloat16* dst) {
  if (jobs.empty()) return TCI_OK;
  Job* dj = nullptr;
  TCI_TRY(tci_dev_alloc(ctx, sizeof(Job) * jobs.size(), (void**)&dj));
  cudaError_t e = cudaMemcpyAsync(dj, jobs.data(), sizeof(Job) * jobs.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (max_work + 255) / 256)), (unsigned)jobs.size());
    kern<<<grid, 256, 0, ctx->stream>>>(dj, src, dst);
    e = cudaStreamSynchronize(ctx->stream);
  }
  tci_dev_free(dj);
  if (e != cudaSuccess) return tci_cuda_fail(ctx, e, "block-sparse pack");
  return TCI_OK;
}

// W.W task over a sector pair (ja, ib): inputs U[(a', t), (b, wr)] for the
// (t, wr) that exist; outputs V[(s, b), (wl, a')] for the (wl, s) that exist.
struct WWTask {
  const float* u[4 * BS_DW];   // element (a'=0, b=0) of input (t, wr), or null
  int64_t ldu[4 * BS_DW];
  int64_t v[4 * BS_DW];        // bf16 element offset of output (wl, s) (b=0, a'=0) in plane 0, or -1
  int64_t ldv[4 * BS_DW];      // row stride (b -> b+1) of that output
  int64_t plane[4 * BS_DW];    // plane stride of that output's piece buffer
  int64_t na, nb;              // sector dims of a' (ja) and b (ib)
};

static_assert(sizeof(WWTask) % sizeof(int64_t) == 0, "WWTask is copied as int64 words");

struct WWCoef {
  float ww[BS_DW * 4 * BS_DW * 4];   // [wl][s][wr][t]
};

// The nonzero W.W coefficients by output (wl, s): terms [start[o], start[o+1])
// multiply input q[k] = t * Dw + wr by c[k] (the Heisenberg MPO has 30 of 400).
// used: bit q set when input q enters some term.
struct WWSparse {
  float c[BS_DW * 4 * BS_DW * 4];
  unsigned char q[BS_DW * 4 * BS_DW * 4];
  unsigned char start[4 * BS_DW + 1];
  unsigned int used;
};

WWSparse ww_sparse(const WWCoef& w) {
  WWSparse sp;
  memset(&sp, 0, sizeof sp);
  int k = 0;
  for (int o = 0; o < 4 * BS_DW; ++o) {
    sp.start[o] = (unsigned char)k;
    for (int wr = 0; wr < BS_DW; ++wr)
      for (int t = 0; t < 4; ++t) {
        const float c = w.ww[(o * BS_DW + wr) * 4 + t];
        if (c == 0.f) continue;
        sp.c[k] = c;
        sp.q[k] = (unsigned char)(t * BS_DW + wr);
        sp.used |= 1u << (t * BS_DW + wr);
        ++k;
      }
  }
  sp.start[4 * BS_DW] = (unsigned char)k;
  return sp;
}

struct WWTile {
  int task;
  int a0, b0;
};

// Variant 0: one block per (task, 32 a' x 8 b tile).  The tile of every
// existing input (t, wr) that some coefficient uses is staged in shared memory
// with row reads of 8 contiguous b, then each thread forms the outputs of one
// (a', b) pair from the nonzero coefficients only and writes them with a'
// fastest (contiguous along GEMM2's K dimension).
constexpr int kWA = 32, kWB = 8;

__global__ void __launch_bounds__(kWA * kWB) k_bs_ww(const WWTask* __restrict__ tasks, const WWTile* __restrict__ tiles,
                                                     const WWSparse sp, __nv_bfloat16* __restrict__ V) {
  __shared__ float Us[4 * BS_DW][kWA][kWB + 1];
  __shared__ WWTask T;   // the task's pointers and strides, read once per block
  const WWTile tl = tiles[blockIdx.x];
  {
    const int64_t* src = (const int64_t*)&tasks[tl.task];
    int64_t* dst = (int64_t*)&T;
    for (int i = threadIdx.x; i < (int)(sizeof(WWTask) / sizeof(int64_t)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int na = (int)T.na, nb = (int)T.nb;
  {
    const int bl = threadIdx.x % kWB, al = threadIdx.x / kWB;
    const int ap = tl.a0 + al, b = tl.b0 + bl;
    const bool in = ap < na && b < nb;
    for (int q = 0; q < 4 * BS_DW; ++q) {   // uniform: only inputs some coefficient uses
      if (!((sp.used >> q) & 1u)) continue;
      const float* u = T.u[q];
      Us[q][al][bl] = (u && in) ? u[ap * (int)T.ldu[q] + b] : 0.f;
    }
  }
  __syncthreads();
  const int al = threadIdx.x % kWA, bl = threadIdx.x / kWA;
  const int ap = tl.a0 + al, b = tl.b0 + bl;
  if (ap >= na || b >= nb) return;
  for (int o = 0; o < 4 * BS_DW; ++o) {
    const int k0 = sp.start[o], k1 = sp.start[o + 1];
    if (k0 == k1 || T.v[o] < 0) continue;
    float acc = 0.f;
    for (int k = k0; k < k1; ++k) acc = fmaf(sp.c[k], Us[sp.q[k]][al][bl], acc);
    const __nv_bfloat16 h = __float2bfloat16_rn(acc);
    const float r1 = acc - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
    __nv_bfloat16* vo = V + T.v[o] + (b * (int)T.ldv[o] + ap);
    const int64_t pl = T.plane[o];
    vo[0] = h;
    vo[pl] = m;
    vo[2 * pl] = l;
  }
}

// Variants 1-3: one thread per 4 a' x 4 b micro-tile and group of outputs
// (outputs o = blockIdx.y, + gridDim.y, ...: 1, 4 or 10 groups, so that more
// threads each run a shorter chain of dependent loads), one block per (task,
// 64 a' x 32 b tile, output group); no shared memory.  For each output (wl, s) the thread
// reads its inputs' micro-tiles as 16-byte rows (U sub-blocks start on
// 16-byte boundaries and their rows are padded to 4), forms the 16 sums with
// the terms in the same order as variant 0 (so the results are identical),
// and writes each b row's 4 a' as one 8-byte vector per piece plane (V
// sub-blocks start on 4-element K offsets).  Rows a' >= na read nothing and
// write zeros, which land in the zero K padding after the sub-block; columns
// b >= nb (read from the padded row) are not written.
constexpr int kW4A = 16, kW4B = 8;   // micro-tiles per block along a' and b (128 threads)
constexpr int kWVariants = 4;
constexpr int kWGroups[kWVariants] = {0, 1, 4, 10};   // output groups of variants 1-3

__device__ __forceinline__ uint2 pack4_bf16(float x0, float x1, float x2, float x3) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(x0, x1), hi = __floats2bfloat162_rn(x2, x3);
  return make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
}

__global__ void __launch_bounds__(kW4A * kW4B) k_bs_ww4(const WWTask* __restrict__ tasks,
                                                        const WWTile* __restrict__ tiles, const WWSparse sp,
                                                        __nv_bfloat16* __restrict__ V) {
  const WWTile tl = tiles[blockIdx.x];
  const WWTask* __restrict__ T = tasks + tl.task;
  const int na = (int)T->na, nb = (int)T->nb;
  const int a0 = tl.a0 + 4 * (threadIdx.x % kW4A), b0 = tl.b0 + 4 * (threadIdx.x / kW4A);
  if (a0 >= na || b0 >= nb) return;
  for (int o = blockIdx.y; o < 4 * BS_DW; o += gridDim.y) {
    const int k0 = sp.start[o], k1 = sp.start[o + 1];
    const int64_t vofs = T->v[o];
    if (k0 == k1 || vofs < 0) continue;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k = k0; k < k1; ++k) {
      const int q = sp.q[k];
      const float* u = T->u[q];
      const float c = sp.c[k];
      const int ld = (int)T->ldu[q];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        // a missing input (or a row past na) contributes c * 0, as in variant 0
        const float4 x = (u && a0 + i < na) ? __ldg(reinterpret_cast<const float4*>(u + (a0 + i) * ld + b0))
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
        acc[i][0] = fmaf(c, x.x, acc[i][0]);
        acc[i][1] = fmaf(c, x.y, acc[i][1]);
        acc[i][2] = fmaf(c, x.z, acc[i][2]);
        acc[i][3] = fmaf(c, x.w, acc[i][3]);
      }
    }
    const int ldv = (int)T->ldv[o];
    const int64_t pl = T->plane[o];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (b0 + j >= nb) break;
      float h[4], m[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float x = acc[i][j];
        h[i] = __bfloat162float(__float2bfloat16_rn(x));
        const float r1 = x - h[i];
        m[i] = __bfloat162float(__float2bfloat16_rn(r1));
        l[i] = r1 - m[i];
      }
      __nv_bfloat16* vp = V + vofs + ((b0 + j) * ldv + a0);
      *reinterpret_cast<uint2*>(vp) = pack4_bf16(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint2*>(vp + pl) = pack4_bf16(m[0], m[1], m[2], m[3]);
      *reinterpret_cast<uint2*>(vp + 2 * pl) = pack4_bf16(l[0], l[1], l[2], l[3]);
    }
  }
}

__global__ void k_bs_ww_precompute(const double* __restrict__ W, float* __restrict__ out) {
  // out[((wl*4 + s1*2+s2)*Dw + wr)*4 + t1*2+t2] = sum_wm W[wl,wm,s1,t1] W[wm,wr,s2,t2]
  for (int i = threadIdx.x; i < BS_DW * 4 * BS_DW * 4; i += blockDim.x) {
    int r = i;
    const int t = r % 4; r /= 4;
    const int wr = r % BS_DW; r /= BS_DW;
    const int s = r % 4; r /= 4;
    const int wl = r;
    const int s1 = s / 2, s2 = s % 2, t1 = t / 2, t2 = t % 2;
    double acc = 0.0;
    for (int wm = 0; wm < BS_DW; ++wm)
      acc += W[((wl * BS_DW + wm) * 2 + s1) * 2 + t1] * W[((wm * BS_DW + wr) * 2 + s2) * 2 + t2];
    out[i] = (float)acc;
  }
}

}  // namespace

struct tci_bs_plan_s {
  int magic;
  tci_context ctx;
  int products, chunk_k, xchunk_k;
  int raster = 0;
  int64_t psi_elems;          // packed psi/out element count
  double flops;               // algorithmic flops of one matvec
  // device buffers
  void* arena = nullptr;      // bf16 pieces: psi blocks, Rg, Lg, Vg
  float* U = nullptr;         // GEMM1 outputs
  float* out_stage = nullptr; // GEMM2 writes here (the group table holds fixed pointers)
  SplitJob* d_psi_jobs = nullptr;
  UnpackJob* d_unpack = nullptr;   // staged GEMM2 result -> packed output blocks
  BsChunk* d_split_chunks = nullptr;
  BsChunk* d_unpack_chunks = nullptr;
  int n_unpack = 0, n_split_chunks = 0, n_unpack_chunks = 0;
  WWTask* d_tasks = nullptr;
  WWTile* d_tiles[2] = {nullptr, nullptr};   // per W.W variant
  int n_tiles[2] = {0, 0};
  int ww_var = 2;                            // W.W kernel variant (tuned)
  int n_psi_jobs = 0, n_tasks = 0;
  int64_t max_task_elems = 0;
  tci_split_group* g1 = nullptr;     // 128-wide tiles
  tci_split_group* g2 = nullptr;
  tci_split_group* g1n = nullptr;    // 64-wide tiles (a tile shape the autotuner may choose)
  tci_split_group* g2n = nullptr;
  int bn = 128;
  WWCoef coef;
  WWSparse ww_sp;   // the nonzero coefficients (the W.W kernel's argument)
  int64_t n_gemm1 = 0, n_gemm2 = 0;
  double tensor_flops = 0.0;
  tci_graph graph;              // captured split -> GEMM1 -> W.W -> GEMM2
  const float* cap_psi = nullptr;
  float* cap_out = nullptr;     // the unpack's destination (null: stop after GEMM2, e.g. while tuning)
};

struct BsBlock {
  int i, a, b, j;      // psi: (ia, t1, t2, ib); env: (i, w, -, j)
  int64_t off;         // element offset in the packed buffer
};

extern "C" tci_status tci_bs_heff_plan_create(tci_context ctx, int nsec, const int32_t* sector_charge,
                                              const int64_t* sector_dim, const int32_t* phys_charge,
                                              const int32_t* mpo_charge, const float* L_packed,
                                              const float* R_packed, const double* W, tci_bs_plan* out) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "bs_heff_plan_create");
  if (!out) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs_heff_plan_create: NULL output");
  *out = nullptr;
  if (nsec <= 0 || !sector_charge || !sector_dim || !phys_charge || !mpo_charge || !L_packed || !R_packed || !W)
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs_heff_plan_create: NULL argument or no sectors");
  if (ctx->precision == TCI_PREC_NATIVE)
    return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "bs_heff_plan_create: the block-sparse path runs in a split precision");
  std::map<int, int> idx;
  for (int i = 0; i < nsec; ++i) {
    if (sector_dim[i] <= 0) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs_heff_plan_create: sector dims must be positive");
    if (idx.count(sector_charge[i])) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs_heff_plan_create: repeated sector charge");
    idx[sector_charge[i]] = i;
  }
  auto sec = [&](int q) {
    auto it = idx.find(q);
    return it == idx.end() ? -1 : it->second;
  };
  const int64_t* dim = sector_dim;
  // ---------------------------------------------------------------- block lists
  std::vector<BsBlock> P, Lb, Rb;   // psi, L, R
  std::map<long, int> Pidx, Lidx, Ridx;
  int64_t off = 0;
  for (int ia = 0; ia < nsec; ++ia)
    for (int t1 = 0; t1 < BS_D; ++t1)
      for (int t2 = 0; t2 < BS_D; ++t2) {
        const int ib = sec(sector_charge[ia] + phys_charge[t1] + phys_charge[t2]);
        if (ib < 0) continue;
        Pidx[((long)ia * 4 + t1 * 2 + t2) * 4096 + ib] = (int)P.size();
        P.push_back({ia, t1, t2, ib, off});
        off += dim[ia] * dim[ib];
      }
  const int64_t psi_elems = off;
  off = 0;
  for (int ia = 0; ia < nsec; ++ia)
    for (int w = 0; w < BS_DW; ++w) {
      const int j = sec(sector_charge[ia] + mpo_charge[w]);
      if (j < 0) continue;
      Lidx[((long)ia * BS_DW + w)] = (int)Lb.size();
      Lb.push_back({ia, w, 0, j, off});
      off += dim[ia] * dim[j];
    }
  Rb = Lb;   // same structure and packed offsets
  for (auto& kv : Lidx) Ridx[kv.first] = kv.second;

  tci_bs_plan p = new tci_bs_plan_s();
  p->magic = kBsMagic;
  p->ctx = ctx;
  p->products = ctx->precision == TCI_PREC_SPLIT_BF16_3 ? 3 : 6;
  p->chunk_k = ctx->split_chunk_k;
  p->xchunk_k = ctx->split_xchunk_k;
  p->psi_elems = psi_elems;
  auto fail = [&](tci_status s) {
    tci_bs_plan pp = p;
    tci_bs_plan_destroy(&pp);
    return s;
  };

  // ---------------------------------------------------------------- arena layout
  // Rg[ib'] : rows (wr, b) over R blocks (ib(wr), wr, ib'), K = dim[ib']
  struct Stack {
    int64_t rows = 0, K = 0, Kp = 0, off = 0;   // off: bf16 elements (plane 0)
    std::vector<int64_t> row_off;               // per w (or -1)
    std::vector<int> blk;                       // block per w (or -1)
  };
  std::vector<Stack> Rg(nsec), Lg(nsec);
  int64_t arena = 0;   // in bf16 elements, each buffer 256-byte aligned
  auto take = [&](int64_t elems) {
    const int64_t o = arena;
    arena += al256(elems * 2) / 2;
    return o;
  };
  std::vector<SliceJob> init_jobs_R;
  for (int jb = 0; jb < nsec; ++jb) {
    Stack& S = Rg[jb];
    S.row_off.assign(BS_DW, -1);
    S.blk.assign(BS_DW, -1);
    S.K = dim[jb];
    S.Kp = pad8(S.K);
    for (int w = 0; w < BS_DW; ++w) {
      const int ib = sec(sector_charge[jb] - mpo_charge[w]);   // R block (ib, w, jb): q_jb = q_ib + Delta(w)
      if (ib < 0) continue;
      S.row_off[w] = S.rows;
      S.blk[w] = Ridx[(long)ib * BS_DW + w];
      S.rows = pad4(S.rows + dim[ib]);   // every U sub-block starts on a 16-byte boundary
    }
    if (S.rows) S.off = take(3 * S.rows * S.Kp);
    for (int w = 0; w < BS_DW; ++w)
      if (S.blk[w] >= 0) {
        // rows of R block (ib, w, jb) -> rows [row_off[w], + dim ib) of every plane of the stack
        const BsBlock& B = Rb[S.blk[w]];
        init_jobs_R.push_back({B.off, dim[B.i], S.K, S.K, S.off + S.row_off[w] * S.Kp, S.Kp, S.rows * S.Kp});
      }
  }
  for (int ia = 0; ia < nsec; ++ia) {
    Stack& S = Lg[ia];
    S.row_off.assign(BS_DW, -1);   // here: K offset of each wl
    S.blk.assign(BS_DW, -1);
    S.rows = dim[ia];
    for (int w = 0; w < BS_DW; ++w) {
      auto it = Lidx.find((long)ia * BS_DW + w);
      if (it == Lidx.end()) continue;
      S.row_off[w] = S.K;
      S.blk[w] = it->second;
      S.K = pad4(S.K + dim[Lb[it->second].j]);   // every V sub-block starts on an 8-byte boundary
    }
    S.Kp = pad8(S.K);
    if (S.K) S.off = take(3 * S.rows * S.Kp);
  }
  // psi pieces stacked per sector ib' (GEMM1's A operand): [3][sum of dim ia'][pad8(dim ib')],
  // block k at rows [prow[k], + dim ia') of every plane
  std::vector<int64_t> pstack_rows(nsec, 0), pstack_off(nsec, 0), prow(P.size());
  for (size_t k = 0; k < P.size(); ++k) {
    prow[k] = pstack_rows[P[k].j];
    pstack_rows[P[k].j] += dim[P[k].i];
  }
  for (int j = 0; j < nsec; ++j)
    if (pstack_rows[j]) pstack_off[j] = take(3 * pstack_rows[j] * pad8(dim[j]));
  std::vector<SplitJob> psi_jobs;
  for (size_t k = 0; k < P.size(); ++k) {
    const BsBlock& B = P[k];
    const int64_t K = dim[B.j], Kp = pad8(K);
    psi_jobs.push_back({B.off, dim[B.i], K, K, Kp, pstack_off[B.j] + prow[k] * Kp, pstack_rows[B.j] * Kp});
  }
  // Vg stacked per sector ia (GEMM2's B operand): [3][sum of dim ib][Lg[ia].Kp],
  // output block k at rows [vcol[k], + dim ib) of every plane
  std::vector<int64_t> vstack_rows(nsec, 0), vstack_off(nsec, 0), vcol(P.size());
  for (size_t k = 0; k < P.size(); ++k) {
    vcol[k] = vstack_rows[P[k].i];
    vstack_rows[P[k].i] += dim[P[k].j];
  }
  for (int ia = 0; ia < nsec; ++ia)
    if (vstack_rows[ia] && Lg[ia].K) vstack_off[ia] = take(3 * vstack_rows[ia] * Lg[ia].Kp);
  // U stacked like psi: [sum of dim ia'][pad4(Rg[ib'].rows)] FP32 per sector ib'
  std::vector<int64_t> ustack_off(nsec, 0), Uoff(P.size());
  int64_t uelems = 0;
  for (int j = 0; j < nsec; ++j)
    if (pstack_rows[j] && Rg[j].rows) {
      ustack_off[j] = uelems;
      uelems += al256(pstack_rows[j] * pad4(Rg[j].rows) * 4) / 4;
    }
  for (size_t k = 0; k < P.size(); ++k) Uoff[k] = ustack_off[P[k].j] + prow[k] * pad4(Rg[P[k].j].rows);
  tci_status s;
  if ((s = tci_dev_alloc(ctx, std::max<int64_t>(arena, 8) * 2, &p->arena)) != TCI_OK) return fail(s);
  if ((s = tci_dev_alloc(ctx, std::max<int64_t>(uelems, 1) * 4, (void**)&p->U)) != TCI_OK) return fail(s);
  __nv_bfloat16* A = (__nv_bfloat16*)p->arena;
  cudaError_t e = cudaMemsetAsync(p->arena, 0, std::max<int64_t>(arena, 8) * 2, ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan memset"));

  // ---------------------------------------------------------------- pack R and L pieces (once)
  {
    int64_t mx = 0;
    for (auto& j : init_jobs_R) mx = std::max(mx, j.rows * j.K);
    if ((s = run_jobs<SliceJob>(ctx, init_jobs_R, mx, k_bs_split_slice, R_packed, A)) != TCI_OK) return fail(s);
    std::vector<SliceJob> lj;
    mx = 0;
    for (int ia = 0; ia < nsec; ++ia) {
      const Stack& S = Lg[ia];
      for (int w = 0; w < BS_DW; ++w)
        if (S.blk[w] >= 0) {
          const BsBlock& B = Lb[S.blk[w]];
          lj.push_back({B.off, dim[ia], dim[B.j], dim[B.j], S.off + S.row_off[w], S.Kp, S.rows * S.Kp});
          mx = std::max(mx, dim[ia] * dim[B.j]);
        }
    }
    if ((s = run_jobs<SliceJob>(ctx, lj, mx, k_bs_split_slice, L_packed, A)) != TCI_OK) return fail(s);
  }

  // ---------------------------------------------------------------- GEMM1 group
  std::vector<tci_split_problem> g1;
  for (int j = 0; j < nsec; ++j) {
    const Stack& S = Rg[j];
    if (!S.rows || !pstack_rows[j]) continue;
    g1.push_back({A + pstack_off[j], A + S.off, pstack_rows[j], S.rows, S.Kp, p->U + ustack_off[j], 1, pad4(S.rows), 1});
  }
  for (auto& q : g1) p->tensor_flops += 2.0 * p->products * q.M * q.N * q.Kp;
  if ((s = tci_split_group_create(ctx, (int)g1.size(), g1.data(), &p->g1, 128)) != TCI_OK) return fail(s);
  if ((s = tci_split_group_create(ctx, (int)g1.size(), g1.data(), &p->g1n, 64)) != TCI_OK) return fail(s);
  p->n_gemm1 = (int64_t)g1.size();
  // ---------------------------------------------------------------- W.W tasks
  std::map<long, int> task_of;   // (ja, ib) -> task
  std::vector<WWTask> tasks;
  auto task = [&](int ja, int ib) -> WWTask& {
    const long key = (long)ja * 4096 + ib;
    auto it = task_of.find(key);
    if (it != task_of.end()) return tasks[it->second];
    WWTask T;
    memset(&T, 0, sizeof T);
    for (int q = 0; q < 4 * BS_DW; ++q) T.v[q] = -1;
    T.na = dim[ja];
    T.nb = dim[ib];
    task_of[key] = (int)tasks.size();
    tasks.push_back(T);
    return tasks.back();
  };
  for (size_t k = 0; k < P.size(); ++k) {           // inputs
    const BsBlock& B = P[k];                        // (ja, t1, t2, ib')
    const Stack& S = Rg[B.j];
    const int t = B.a * 2 + B.b;
    for (int wr = 0; wr < BS_DW; ++wr) {
      if (S.blk[wr] < 0) continue;
      const int ib = Rb[S.blk[wr]].i;
      WWTask& T = task(B.i, ib);
      T.u[t * BS_DW + wr] = p->U + Uoff[k] + S.row_off[wr];
      T.ldu[t * BS_DW + wr] = pad4(S.rows);
    }
  }
  for (size_t k = 0; k < P.size(); ++k) {           // outputs
    const BsBlock& O = P[k];                        // (ia, s1, s2, ib)
    const Stack& S = Lg[O.i];
    const int sidx = O.a * 2 + O.b;
    for (int wl = 0; wl < BS_DW; ++wl) {
      if (S.blk[wl] < 0) continue;
      const int ja = Lb[S.blk[wl]].j;
      auto it = task_of.find((long)ja * 4096 + O.j);
      if (it == task_of.end()) continue;            // no U feeds this V sub-block: it stays zero
      WWTask& T = tasks[it->second];
      T.v[wl * 4 + sidx] = vstack_off[O.i] + vcol[k] * S.Kp + S.row_off[wl];
      T.ldv[wl * 4 + sidx] = S.Kp;
      T.plane[wl * 4 + sidx] = vstack_rows[O.i] * S.Kp;
    }
  }
  p->n_tasks = (int)tasks.size();
  for (auto& T : tasks) {
    p->max_task_elems = std::max(p->max_task_elems, T.na * T.nb);
    for (int q = 0; q < 4 * BS_DW; ++q)   // the W.W kernel's 32-bit offsets inside a task
      if ((T.u[q] && T.na * T.ldu[q] + T.nb >= ((int64_t)1 << 31)) ||
          (T.v[q] >= 0 && T.nb * T.ldv[q] + T.na >= ((int64_t)1 << 31)))
        return fail(tci_fail(ctx, TCI_ERR_UNSUPPORTED, "bs_heff_plan_create: sector blocks exceed 32-bit offsets"));
  }
  if (!tasks.empty()) {
    if ((s = tci_dev_alloc(ctx, sizeof(WWTask) * tasks.size(), (void**)&p->d_tasks)) != TCI_OK) return fail(s);
    e = cudaMemcpyAsync(p->d_tasks, tasks.data(), sizeof(WWTask) * tasks.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan: tasks"));
    for (int ri = 0; ri < 2; ++ri) {
      const int ta = ri ? 4 * kW4A : kWA, tb = ri ? 4 * kW4B : kWB;
      std::vector<WWTile> wtiles;
      for (int t = 0; t < (int)tasks.size(); ++t)
        for (int64_t a0 = 0; a0 < tasks[t].na; a0 += ta)
          for (int64_t b0 = 0; b0 < tasks[t].nb; b0 += tb) wtiles.push_back({t, (int)a0, (int)b0});
      p->n_tiles[ri] = (int)wtiles.size();
      if ((s = tci_dev_alloc(ctx, sizeof(WWTile) * wtiles.size(), (void**)&p->d_tiles[ri])) != TCI_OK) return fail(s);
      e = cudaMemcpyAsync(p->d_tiles[ri], wtiles.data(), sizeof(WWTile) * wtiles.size(), cudaMemcpyHostToDevice,
                          ctx->stream);
      if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan: W.W tiles"));
    }
  }
  // ---------------------------------------------------------------- GEMM2 group
  // the group table holds fixed pointers: GEMM2 writes the plan's staging
  // buffer, [dim ia][pad4(sum of dim ib)] row-major per sector ia, and the
  // unpack pass writes the caller's output blocks
  std::vector<int64_t> ostage_off(nsec, -1);
  int64_t ost = 0;
  for (int ia = 0; ia < nsec; ++ia)
    if (vstack_rows[ia] && Lg[ia].K) {
      ostage_off[ia] = ost;
      ost += dim[ia] * pad4(vstack_rows[ia]);
    }
  if ((s = tci_dev_alloc(ctx, std::max<int64_t>(ost, 1) * 4, (void**)&p->out_stage)) != TCI_OK) return fail(s);
  std::vector<tci_split_problem> g2;
  for (int ia = 0; ia < nsec; ++ia) {
    const Stack& S = Lg[ia];
    if (ostage_off[ia] < 0) continue;
    g2.push_back({A + S.off, A + vstack_off[ia], dim[ia], vstack_rows[ia], S.Kp, p->out_stage + ostage_off[ia], 1,
                  pad4(vstack_rows[ia]), 1});
  }
  std::vector<UnpackJob> unpack;
  for (size_t k = 0; k < P.size(); ++k) {
    const BsBlock& O = P[k];
    const int64_t so = ostage_off[O.i];
    unpack.push_back({so >= 0 ? so + vcol[k] : -1, pad4(vstack_rows[O.i]), dim[O.i], dim[O.j], O.off});
  }
  p->n_unpack = (int)unpack.size();
  std::vector<BsChunk> uchunks;
  for (size_t k = 0; k < unpack.size(); ++k) {
    const int64_t n = unpack[k].rows * unpack[k].cols;
    if (n >= ((int64_t)1 << 31) - kUnpackElems)
      return fail(tci_fail(ctx, TCI_ERR_UNSUPPORTED, "bs_heff_plan_create: output block exceeds 32-bit offsets"));
    for (int64_t st = 0; st < n; st += kUnpackElems) uchunks.push_back({(int)k, (int)st});
  }
  p->n_unpack_chunks = (int)uchunks.size();
  if (!uchunks.empty()) {
    if ((s = tci_dev_alloc(ctx, sizeof(BsChunk) * uchunks.size(), (void**)&p->d_unpack_chunks)) != TCI_OK)
      return fail(s);
    e = cudaMemcpyAsync(p->d_unpack_chunks, uchunks.data(), sizeof(BsChunk) * uchunks.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan: unpack chunks"));
  }
  if (!unpack.empty()) {
    if ((s = tci_dev_alloc(ctx, sizeof(UnpackJob) * unpack.size(), (void**)&p->d_unpack)) != TCI_OK) return fail(s);
    e = cudaMemcpyAsync(p->d_unpack, unpack.data(), sizeof(UnpackJob) * unpack.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan: unpack jobs"));
  }
  for (auto& q : g2) p->tensor_flops += 2.0 * p->products * q.M * q.N * q.Kp;
  if ((s = tci_split_group_create(ctx, (int)g2.size(), g2.data(), &p->g2, 128)) != TCI_OK) return fail(s);
  if ((s = tci_split_group_create(ctx, (int)g2.size(), g2.data(), &p->g2n, 64)) != TCI_OK) return fail(s);
  p->n_gemm2 = (int64_t)g2.size();
  // psi split jobs
  p->n_psi_jobs = (int)psi_jobs.size();
  std::vector<BsChunk> schunks;
  for (size_t k = 0; k < psi_jobs.size(); ++k) {
    const SplitJob& J = psi_jobs[k];
    // the split writes 16-byte piece vectors: rows, planes and the stack base on 8-element boundaries
    if (J.Kp % 8 || J.plane % 8 || J.dst_off % 8)
      return fail(tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs_heff_plan_create: misaligned psi piece stack"));
    const int64_t n = J.rows * (J.Kp / 8);
    if (n >= ((int64_t)1 << 31) - kSplitOctets)
      return fail(tci_fail(ctx, TCI_ERR_UNSUPPORTED, "bs_heff_plan_create: psi block exceeds 32-bit offsets"));
    for (int64_t st = 0; st < n; st += kSplitOctets) schunks.push_back({(int)k, (int)st});
  }
  p->n_split_chunks = (int)schunks.size();
  if (!schunks.empty()) {
    if ((s = tci_dev_alloc(ctx, sizeof(BsChunk) * schunks.size(), (void**)&p->d_split_chunks)) != TCI_OK)
      return fail(s);
    e = cudaMemcpyAsync(p->d_split_chunks, schunks.data(), sizeof(BsChunk) * schunks.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan: split chunks"));
  }
  if (!psi_jobs.empty()) {
    if ((s = tci_dev_alloc(ctx, sizeof(SplitJob) * psi_jobs.size(), (void**)&p->d_psi_jobs)) != TCI_OK) return fail(s);
    e = cudaMemcpyAsync(p->d_psi_jobs, psi_jobs.data(), sizeof(SplitJob) * psi_jobs.size(),
                        cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan: psi jobs"));
  }
  // W.W coefficients (FP64 product on the device, FP32 copy for the kernel arguments)
  {
    float* d = nullptr;
    if ((s = tci_dev_alloc(ctx, sizeof(WWCoef), (void**)&d)) != TCI_OK) return fail(s);
    k_bs_ww_precompute<<<1, 256, 0, ctx->stream>>>(W, d);
    e = cudaMemcpyAsync(p->coef.ww, d, sizeof(WWCoef), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    tci_dev_free(d);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan: W.W"));
    p->ww_sp = ww_sparse(p->coef);
  }
  // ---------------------------------------------------------------- algorithmic flops
  {
    double fl = 0.0;
    std::map<long, int> ublk;   // sector pairs (ja, ib) carrying U
    for (size_t k = 0; k < P.size(); ++k) {
      const BsBlock& B = P[k];
      const Stack& S = Rg[B.j];
      for (int w = 0; w < BS_DW; ++w)
        if (S.blk[w] >= 0) {
          const int ib = Rb[S.blk[w]].i;
          fl += 2.0 * dim[B.i] * dim[ib] * dim[B.j];
          ublk[(long)B.i * 4096 + ib] = 1;
        }
    }
    for (auto& kv : ublk) fl += 2.0 * dim[kv.first / 4096] * dim[kv.first % 4096] * 16.0 * BS_DW * BS_DW;
    for (size_t k = 0; k < P.size(); ++k) {
      const BsBlock& O = P[k];
      const Stack& S = Lg[O.i];
      for (int w = 0; w < BS_DW; ++w)
        if (S.blk[w] >= 0) {
          const int ja = Lb[S.blk[w]].j;
          if (ublk.count((long)ja * 4096 + O.j)) fl += 2.0 * dim[O.i] * dim[O.j] * dim[ja];
        }
    }
    p->flops = fl;
  }
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "bs plan"));
  vs.info = "blocks=" + std::to_string(P.size()) + " gemm1=" + std::to_string(p->n_gemm1) +
            " gemm2=" + std::to_string(p->n_gemm2) + " ww_tasks=" + std::to_string(p->n_tasks);
  *out = p;
  return TCI_OK;
}

extern "C" tci_status tci_bs_plan_destroy(tci_bs_plan* pp) {
  if (!pp || !*pp || (*pp)->magic != kBsMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "bs_plan_destroy: invalid plan");
  tci_bs_plan p = *pp;
  if (tci_ctx_ok(p->ctx)) cudaStreamSynchronize(p->ctx->stream);
  tci_graph_destroy(&p->graph);
  tci_split_group_destroy(p->g1);
  tci_split_group_destroy(p->g2);
  tci_split_group_destroy(p->g1n);
  tci_split_group_destroy(p->g2n);
  void* bufs[] = {p->arena, p->U, p->out_stage, p->d_psi_jobs, p->d_tasks, p->d_tiles[0], p->d_tiles[1],
                  p->d_unpack, p->d_split_chunks, p->d_unpack_chunks};
  for (void* b : bufs) tci_dev_free(b);
  p->magic = 0;
  delete p;
  *pp = nullptr;
  return TCI_OK;
}

extern "C" double tci_bs_heff_flops(tci_bs_plan p) {
  if (!p || p->magic != kBsMagic) return 0.0;
  return p->flops;
}

extern "C" int64_t tci_bs_psi_size(tci_bs_plan p) {
  if (!p || p->magic != kBsMagic) return -1;
  return p->psi_elems;
}

static tci_status launch_ww(tci_bs_plan p) {
  const int v = p->ww_var;
  if (!p->n_tiles[v ? 1 : 0]) return TCI_OK;
  tci_context ctx = p->ctx;
  __nv_bfloat16* V = (__nv_bfloat16*)p->arena;
  if (v == 0)
    k_bs_ww<<<p->n_tiles[0], kWA * kWB, 0, ctx->stream>>>(p->d_tasks, p->d_tiles[0], p->ww_sp, V);
  else
    k_bs_ww4<<<dim3(p->n_tiles[1], kWGroups[v]), kW4A * kW4B, 0, ctx->stream>>>(p->d_tasks, p->d_tiles[1], p->ww_sp, V);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

static tci_status launch_unpack(tci_bs_plan p, float* out) {
  if (!p->n_unpack_chunks) return TCI_OK;
  k_bs_unpack<<<p->n_unpack_chunks, 256, 0, p->ctx->stream>>>(p->d_unpack_chunks, p->d_unpack, p->out_stage, out);
  TCI_CUDA(p->ctx, cudaGetLastError());
  return TCI_OK;
}

static tci_status bs_launch_all(void* arg) {
  tci_bs_plan p = (tci_bs_plan)arg;
  tci_context ctx = p->ctx;
  if (!p->cap_psi) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs matvec: no input set");
  if (p->n_split_chunks)
    k_bs_split<<<p->n_split_chunks, kSplitOctets, 0, ctx->stream>>>(p->d_split_chunks, p->d_psi_jobs, p->cap_psi,
                                                                      (__nv_bfloat16*)p->arena);
  TCI_CUDA(ctx, cudaGetLastError());
  TCI_TRY(tci_split_group_launch(ctx, p->bn == 64 ? p->g1n : p->g1, p->products, p->chunk_k, p->xchunk_k, p->raster));
  TCI_TRY(launch_ww(p));
  TCI_TRY(tci_split_group_launch(ctx, p->bn == 64 ? p->g2n : p->g2, p->products, p->chunk_k, p->xchunk_k, p->raster));
  if (p->cap_out) TCI_TRY(launch_unpack(p, p->cap_out));
  return TCI_OK;
}

extern "C" tci_status tci_bs_heff_apply(tci_bs_plan p, const float* psi, float* out) {
  if (!p || p->magic != kBsMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "bs_heff_apply: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "bs_heff_apply");
  if (!psi || !out) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs_heff_apply: NULL buffer");
  p->cap_psi = psi;
  p->cap_out = out;
  if (!p->n_split_chunks || !p->n_unpack_chunks) return bs_launch_all(p);
  if (!p->graph.exec) {
    // first call: run eagerly (sets kernel attributes), then capture the sequence
    TCI_TRY(bs_launch_all(p));
    return tci_graph_capture(ctx, &p->graph, bs_launch_all, p, {(const void*)k_bs_split, (const void*)k_bs_unpack});
  }
  // replay with this call's psi (the split's input) and out (the unpack's output)
  const BsChunk* schunks = p->d_split_chunks;
  const SplitJob* jobs = p->d_psi_jobs;
  __nv_bfloat16* dst = (__nv_bfloat16*)p->arena;
  const BsChunk* uchunks = p->d_unpack_chunks;
  const UnpackJob* ujobs = p->d_unpack;
  const float* stage = p->out_stage;
  void* sargs[4] = {(void*)&schunks, (void*)&jobs, (void*)&psi, (void*)&dst};
  void* uargs[4] = {(void*)&uchunks, (void*)&ujobs, (void*)&stage, (void*)&out};
  void** argv[2] = {sargs, uargs};
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

// tci_bs_heff_apply with CUDA events between the stages: ms[0..3] = psi split,
// grouped GEMM1, W.W tasks, grouped GEMM2 (+ the unpack pass).  Synchronises.
extern "C" tci_status tci_bs_heff_apply_timed(tci_bs_plan p, const float* psi, float* out, float* ms) {
  if (!p || p->magic != kBsMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "bs_heff_apply_timed: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  if (!psi || !out || !ms) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs_heff_apply_timed: NULL argument");
  cudaEvent_t ev[5];
  for (auto& e : ev) TCI_CUDA(ctx, cudaEventCreate(&e));
  TCI_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream));
  if (p->n_split_chunks)
    k_bs_split<<<p->n_split_chunks, kSplitOctets, 0, ctx->stream>>>(p->d_split_chunks, p->d_psi_jobs, psi,
                                                                      (__nv_bfloat16*)p->arena);
  TCI_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
  TCI_TRY(tci_split_group_launch(ctx, p->bn == 64 ? p->g1n : p->g1, p->products, p->chunk_k, p->xchunk_k, p->raster));
  TCI_CUDA(ctx, cudaEventRecord(ev[2], ctx->stream));
  TCI_TRY(launch_ww(p));
  TCI_CUDA(ctx, cudaEventRecord(ev[3], ctx->stream));
  TCI_TRY(tci_split_group_launch(ctx, p->bn == 64 ? p->g2n : p->g2, p->products, p->chunk_k, p->xchunk_k, p->raster));
  TCI_TRY(launch_unpack(p, out));
  TCI_CUDA(ctx, cudaEventRecord(ev[4], ctx->stream));
  TCI_CUDA(ctx, cudaEventSynchronize(ev[4]));
  for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  for (auto& e : ev) cudaEventDestroy(e);
  return tci_synchronize(ctx);
}

// BF16 tensor flops executed by the two grouped launches (all piece products,
// padded K, full tiles excluded): 2 * products * sum over problems of M N Kp.
extern "C" double tci_bs_tensor_flops(tci_bs_plan p) {
  if (!p || p->magic != kBsMagic) return 0.0;
  return p->tensor_flops;
}

// ---------------------------------------------------------------- autotuning
namespace {
struct BsTuneArg {
  tci_bs_plan p;
  const float* psi;
};
tci_status bs_run_cfg(void* a, const tci_gemm_cfg& cfg) {
  BsTuneArg* t = (BsTuneArg*)a;
  t->p->chunk_k = cfg.chunk_k;
  t->p->xchunk_k = cfg.xchunk_k;
  t->p->raster = cfg.raster;
  t->p->bn = cfg.bn;
  t->p->cap_psi = t->psi;
  t->p->cap_out = nullptr;   // candidates stop after GEMM2: the caller's output is not touched
  return bs_launch_all(t->p);
}
// W.W kernel variant: the tuned matvec sequence (without the unpack) timed
// with each, four rounds of 10 in alternating order after a warm-up, median
// per variant; the lowest-numbered variant within 2 % of the fastest wins.
tci_status tune_ww(tci_bs_plan p) {
  tci_context ctx = p->ctx;
  if (!p->n_tasks) return TCI_OK;
  float* keep_out = p->cap_out;
  p->cap_out = nullptr;
  cudaEvent_t e0, e1;
  TCI_CUDA(ctx, cudaEventCreate(&e0));
  TCI_CUDA(ctx, cudaEventCreate(&e1));
  std::vector<double> rounds[kWVariants];
  tci_status s = TCI_OK;
  for (int v = 0; v < kWVariants && s == TCI_OK; ++v) {
    p->ww_var = v;
    for (int w = 0; w < 5 && s == TCI_OK; ++w) s = bs_launch_all(p);
  }
  for (int round = 0; round < 4 && s == TCI_OK; ++round)
    for (int q = 0; q < kWVariants && s == TCI_OK; ++q) {
      const int v = (round & 1) ? kWVariants - 1 - q : q;
      p->ww_var = v;
      cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < 10 && s == TCI_OK; ++r) s = bs_launch_all(p);
      cudaEventRecord(e1, ctx->stream);
      if (s != TCI_OK) break;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        s = tci_cuda_fail(ctx, e, "bs autotune: W.W");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      rounds[v].push_back(ms / 10.0);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->cap_out = keep_out;
  if (s != TCI_OK) return s;
  double med[kWVariants], best = 1e300;
  for (int v = 0; v < kWVariants; ++v) {
    std::sort(rounds[v].begin(), rounds[v].end());
    med[v] = 0.5 * (rounds[v][1] + rounds[v][2]);
    best = std::min(best, med[v]);
  }
  for (int v = kWVariants - 1; v >= 0; --v)
    if (med[v] <= 1.02 * best) p->ww_var = v;
  return TCI_OK;
}
}  // namespace

extern "C" int tci_bs_ww_variant(tci_bs_plan p) {
  if (!p || p->magic != kBsMagic) return -1;
  return p->ww_var;
}

extern "C" tci_status tci_bs_set_ww_variant(tci_bs_plan p, int variant) {
  if (!p || p->magic != kBsMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "bs_set_ww_variant: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  if (variant < 0 || variant >= kWVariants)
    return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "bs_set_ww_variant: variant 0..%d", kWVariants - 1);
  if (variant != p->ww_var) {
    cudaStreamSynchronize(p->ctx->stream);
    tci_graph_destroy(&p->graph);   // the next apply captures the new sequence
    p->ww_var = variant;
  }
  return TCI_OK;
}

extern "C" tci_status tci_bs_autotune(tci_bs_plan p, const float* psi, int max_chunk_k, int* chosen) {
  if (!p || p->magic != kBsMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "bs_autotune: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "bs_autotune");
  if (!psi) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bs_autotune: NULL psi");
  BsTuneArg arg{p, psi};
  const std::string key = "bs|n" + std::to_string(p->psi_elems) + "|g" + std::to_string(p->n_gemm1) + "," +
                          std::to_string(p->n_gemm2) + "|p" + std::to_string(p->products);
  tci_gemm_cfg best;
  double ms = 0.0;
  TCI_TRY(tci_autotune(ctx, key, max_chunk_k, true, bs_run_cfg, &arg, &best, &ms, true));
  p->chunk_k = best.chunk_k;
  p->xchunk_k = best.xchunk_k;
  p->raster = best.raster;
  p->bn = best.bn;
  p->cap_psi = psi;   // a cached configuration ran no candidate, which would have set it
  TCI_TRY(tune_ww(p));
  tci_graph_destroy(&p->graph);   // the next apply captures the tuned sequence
  if (chosen) {
    chosen[0] = best.chunk_k;
    chosen[1] = best.xchunk_k;
    chosen[2] = best.raster;
  }
  return tci_synchronize(ctx);
}

extern "C" tci_status tci_bs_set_tile_n(tci_bs_plan p, int bn) {
  if (!p || p->magic != kBsMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "bs_set_tile_n: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  if (bn != 64 && bn != 128) return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "bs_set_tile_n: tile width 64 or 128");
  if (bn != p->bn) {
    cudaStreamSynchronize(p->ctx->stream);
    tci_graph_destroy(&p->graph);   // the next apply captures the new sequence
    p->bn = bn;
  }
  return TCI_OK;
}

extern "C" int tci_bs_tile_n(tci_bs_plan p) {
  if (!p || p->magic != kBsMagic) return -1;
  return p->bn;
}
