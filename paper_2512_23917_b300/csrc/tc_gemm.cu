// Split-BF16 tensor-core GEMM for sm_103a (tcgen05 + TMA + TMEM), plus the
// K0 split/pack kernel that feeds it.
//
//   C(m, n) = sum_k A(m, k) B(n, k),   A, B given as three bfloat16 planes
//   (hi, mid, lo) with hi + mid + lo == fl32(x).  The piece products
//   A_i B_j with i + j <= 2 (6 products) or i + j <= 1 (3 products) run on
//   the tensor cores with FP32 accumulation in tensor memory (TMEM).
//
// Accumulation design.  The FP32 accumulator of tcgen05.mma loses about
// 2^-25 of its own magnitude (on average, always towards zero) every time
// an MMA adds into it, so the error of a long accumulation grows linearly
// with the number of MMAs that add into the same large value.  Therefore:
//   * the dominant product hi*hi accumulates alone in D1 and D1 is drained
//     every `chunk_k` of depth (default 256: 16 MMAs per drain, measured
//     4.3e-7 relative error for the chi = 2048 matvec; 128 gives 2.2e-7);
//   * the five small cross products (magnitude ~2^-8 of hi*hi) accumulate
//     in a second accumulator X drained every `xchunk_k` (default 1024);
//   * drained values are summed error-free in FP32 double-float form
//     (TwoSum: hi + lo) held in the epilogue threads' registers, and the
//     result is rounded once when the tile is stored (FP64, FP32, or as a
//     normalised FP32 pair hi + lo for double-float consumers).
// D1 and X are each double-buffered in TMEM (4 x 128 columns), so draining
// one buffer overlaps the MMAs that fill the other.
//
// Structure: persistent CTAs (one per SM), 128 x 128 output tiles, K staged
// 32 deep (one 64-byte swizzled row per operand row and piece) through a
// 4-stage TMA -> mbarrier -> tcgen05.mma pipeline.
//   warp 0      : TMA producer (one lane)
//   warp 1      : TMEM allocator + MMA issuer (one lane issues, the warp
//                 synchronises)
//   warps 2..17 : epilogue; warp w reads TMEM lanes 32*(w%4)..+31 and
//                 columns 32*((w-2)/4)..+31
//   warp 18     : watcher: performs every mbarrier wait of the MMA issuer
//                 (stage landed, accumulator buffers drained) and hands the
//                 k-blocks to warp 1 in groups through named barriers: a
//                 group ends at an odd stage or at a tile's last k-block (so
//                 mostly stage pairs (0,1), (2,3)), one sync per group, the
//                 barrier named by the group's first stage.
// The MMA issuer itself never waits on shared memory inside its loop: while
// the tensor cores stream operands from shared memory, a shared-memory read
// whose result the issuing thread needs stalls it for about as long as the
// MMA queue holds work, so the tensor pipe idled ~200 clocks per k-block
// (measured: 64 -> 80 clocks per 128x128x16 MMA with one mbarrier test per
// 12 MMAs); a named-barrier sync costs far less, and one per stage pair
// instead of one per stage took the chi = 2048 GEMM from 1.55 to 1.40 ms
// (two pairs in flight keep the TMA latency hidden).  A group never spans two
// tiles, so a short tile's last k-block is not held back until the next
// tile's first one lands.
// Named-barrier use cannot deadlock or skew: the MMA warp and the watcher both
// run the CTA's whole tile / k-block sequence (after an abort the MMA warp
// still synchronises and commits each k-block, issuing no MMAs) with the same
// group boundaries, the MMA warp syncing at each group's first k-block and the
// watcher arriving after its last, so the counts match.  Barrier s is used at
// most once per pass over the stages; the watcher's arrival for its use in
// pass r follows its wait for stage s's refill in pass r, which follows the
// MMA warp's commit of stage s in pass r - 1 (full implies empty), so the MMA
// warp has passed every earlier sync on barrier s; after an abort the watcher
// waits for that commit on the stage's empty barrier itself.  Every wait of
// the watcher is bounded.
// Every wait is bounded (2 s, or the context's wait limit); on expiry the
// kernel records a status word, lets its in-flight copies and MMAs land
// (those final drains always allow 2 s), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "ptx_sm100.cuh"
#include <string.h>

#include <algorithm>
#include <vector>

#include "tci_internal.cuh"

namespace {

constexpr int TBM = 128;
constexpr int TBN = 128;
constexpr int TBK = 32;   // bf16 elements = 64 B rows, SWIZZLE_64B
constexpr int PIECE_A = TBM * TBK * 2;   // 8 KB
constexpr int STAGE_A = 3 * PIECE_A;
constexpr int NEPI = 16;                         // epilogue warps (4 per TMEM lane quadrant)
constexpr int kWatchWarp = 2 + NEPI;             // waits on the MMA issuer's barriers for it
constexpr int NTHREADS = 64 + 32 * NEPI + 32;
constexpr int kStageBar = 1;                     // named barrier kStageBar + s hands the group starting at stage s
constexpr int kMaxDots = 24;                     // fused dot products: basis vectors + 1 (sum of squares)
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

// Tile width BN of a launch: 128 (every launch) or 64 (grouped launches of
// narrow problems, a tile shape the autotuner may choose).  The accumulators
// take 4 x BN tensor-memory columns (D1 and X, each double-buffered).  The
// narrow tile's smaller stages buy a deeper operand pipeline (6 stages of
// 36 KB against 4 of 48 KB): short problems are bound by TMA latency.
template <int BN>
struct TileN {
  static_assert(BN == 64 || BN == 128, "tile width 64 or 128");
  static constexpr int kPieceB = BN * TBK * 2;
  static constexpr int kStageB = 3 * kPieceB;
  static constexpr int kStageBytes = STAGE_A + kStageB;
  static constexpr int kStages = BN == 64 ? 6 : 4;   // even: stages are handed over in pairs
  static constexpr int kTmemCols = 4 * BN;
  static constexpr int kCols = BN / (NEPI / 4);
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256 + NEPI * kMaxDots * 8;
  static_assert(kStages % 2 == 0 && 2 * kStages + 9 <= 32, "barrier block holds the stage barriers");
  static_assert(kStageBar + kStages <= 15, "named barrier per group start stage");
  static_assert(kSmem <= 232448, "227 KB of shared memory per CTA");
};

// One GEMM of a (possibly grouped) launch.  In a grouped launch the table
// lives in device memory, sorted by decreasing K so the longest tiles are
// scheduled first; tiles of problem i are [tile_begin, tile_begin + num_m*num_n).
struct GemmProblem {   // aligned as its tensor maps (TMA descriptors in global memory)
  CUtensorMap tmA;   // bf16 pieces [3][M][Kp], box {32, 128, 3}
  CUtensorMap tmB;   // bf16 pieces [3][N][Kp], box {32, 128, 3}
  void* C;
  int64_t M, N, scm, scn;
  int num_m, num_n, num_kb, tile_begin;
  int out_mode, pad0, pad1, pad2;
  // out_mode 3 (gate epilogue, see gate16): the bond dimension and the complex
  // offsets of the bond's gate (16 values) and theta in the launch's buffers
  int64_t g_chi, g_off, th_off;
};
static_assert(alignof(GemmProblem) >= 64 && sizeof(GemmProblem) % 64 == 0, "tensor maps need 64-byte alignment");

struct GemmParams {
  const GemmProblem* table;   // grouped launches only
  const int2* tile_map;       // grouped launches: per tile {problem index, k-blocks} (one load per tile)
  int nprob, num_tiles;
  int raster;                 // 0: m-fastest tile order; G > 0: groups of G m-blocks, n-fastest inside
  int kb_d1, kb_x;            // k-blocks per D1 drain / per X drain (kb_x % kb_d1 == 0)
  int products;
  int* status;
  uint64_t wait_ns;           // limit of every wait on work in flight (the final drains keep WAIT_LIMIT_NS)
  // fused dot products (DOTS; one FP64 problem stored row-major, C[m*N + n]): the
  // epilogue also forms <V_i, C> (i < dot_nv, V_i = dot_V + i*dot_ldv, same flat
  // layout as C) and <C, C> over the tiles it stores; CTA b writes its partial
  // sums to dot_part[i*dot_stride + b] (i = dot_nv for <C, C>)
  const double* dot_V;
  int64_t dot_ldv;
  int dot_nv, dot_stride;
  double* dot_part;
  const float2* const* gate_ptrs;   // out_mode 3: device array {gate base, theta base} (complex64)
};

// Local tile index -> (m-block, n-block).  With raster G > 0, consecutive
// tiles sweep G m-blocks by all n-blocks, so concurrently running CTAs share
// both A rows and B rows in L2.
__device__ __forceinline__ void tile_coords(int lt, int num_m, int num_n, int raster, int& mb, int& nb) {
  if (raster <= 0 || raster >= num_m) {
    mb = lt % num_m;
    nb = lt / num_m;
    return;
  }
  const int per = raster * num_n;
  const int first = (lt / per) * raster;
  const int gsz = min(num_m - first, raster);
  const int r = lt - (lt / per) * per;
  mb = first + r % gsz;
  nb = r / gsz;
}

template <bool G>
__device__ __forceinline__ const GemmProblem* find_problem(int tile, const GemmProblem* single, const GemmParams& p) {
  if (!G) return single;
  return &p.table[__ldg(&p.tile_map[tile].x)];
}

// k-blocks of a tile (the MMA issuer and the watcher need nothing else)
template <bool G>
__device__ __forceinline__ int tile_kblocks(int tile, const GemmProblem* single, const GemmParams& p) {
  if (!G) return single->num_kb;
  return __ldg(&p.tile_map[tile].y);
}

// Gate epilogue of one TEBD bond (theta formation with the gate applied).  The
// tile holds AB = A_i B_i with rows (a, t1) and columns (b, t2, c), c = 0 the
// real and c = 1 the imaginary part, the last index fastest; row (a, 1 - t1)
// sits in the partner lane (lane ^ 1).  For the 4 b of the 16 columns from
// ncol0 (ncol0 % 16 == 0) this thread writes
//   theta[a, s1 = t1, s2, b] = sum_{t1', t2'} G[s1, s2, t1', t2'] AB[a, t1', t2', b].
// Called by whole warps: lanes past the last row exchange values but store nothing.
__device__ __forceinline__ void gate16(const float (&v)[16], int64_t row, int64_t ncol0, const GemmProblem* pr,
                                       const GemmParams& p) {
  float o[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) o[j] = __shfl_xor_sync(0xffffffffu, v[j], 1);
  if (row >= pr->M) return;
  const int64_t chi = pr->g_chi, a = row >> 1, b0 = ncol0 >> 2;
  const int t1 = (int)(row & 1);
  // G[s1][s2][t1'][t2'] as float4 pairs over t2': element s1*4 + s2*2 + t1'
  const float4* gs = reinterpret_cast<const float4*>(p.gate_ptrs[0] + pr->g_off) + t1 * 4;
  float2* th = const_cast<float2*>(p.gate_ptrs[1]) + pr->th_off + (a * 2 + t1) * 2 * chi;
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    const float4 go = __ldg(gs + s2 * 2 + t1);         // t1' = t1 (this lane's row)
    const float4 gp = __ldg(gs + s2 * 2 + (t1 ^ 1));   // t1' = 1 - t1 (the partner's row)
    float2 r[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float* x = v + m * 4;   // (t2' = 0: re, im; t2' = 1: re, im)
      const float* y = o + m * 4;
      float re = go.x * x[0] - go.y * x[1];
      float im = go.x * x[1] + go.y * x[0];
      re = fmaf(go.z, x[2], fmaf(-go.w, x[3], re));
      im = fmaf(go.z, x[3], fmaf(go.w, x[2], im));
      re = fmaf(gp.x, y[0], fmaf(-gp.y, y[1], re));
      im = fmaf(gp.x, y[1], fmaf(gp.y, y[0], im));
      re = fmaf(gp.z, y[2], fmaf(-gp.w, y[3], re));
      im = fmaf(gp.z, y[3], fmaf(gp.w, y[2], im));
      r[m] = make_float2(re, im);
    }
    float2* dst = th + s2 * chi + b0;
    if (b0 + 4 <= chi && (((uintptr_t)dst) & 15) == 0) {
      reinterpret_cast<float4*>(dst)[0] = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
      reinterpret_cast<float4*>(dst)[1] = make_float4(r[2].x, r[2].y, r[3].x, r[3].y);
    } else {
#pragma unroll
      for (int m = 0; m < 4; ++m)
        if (b0 + m < chi) dst[m] = r[m];
    }
  }
}

// Error-free sum in FP32: s + e == a + b exactly (Knuth TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Two columns of the drain fold in packed FP32x2 arithmetic (the same IEEE
// round-to-nearest adds and subtracts as two_sum, two lanes per instruction):
// (s0, s1) + (e0, e1) == (a0 + b0, a1 + b1) exactly, then the compensation pair
// rl (packed bfloat16) += (e0, e1), rounded back to bfloat16.
__device__ __forceinline__ void two_sum2_fold(float& a0, float& a1, uint32_t b0, uint32_t b1, __nv_bfloat162& rl) {
  uint32_t r = *reinterpret_cast<const uint32_t*>(&rl);
  asm("{\n\t"
      ".reg .b64 a, b, s, bp, ap, t1, t2, e, c, q;\n\t"
      ".reg .b32 cx, cy, q0, q1;\n\t"
      "mov.b64 a, {%0, %1};\n\t"
      "mov.b64 b, {%3, %4};\n\t"
      "add.rn.f32x2 s, a, b;\n\t"
      "sub.rn.f32x2 bp, s, a;\n\t"
      "sub.rn.f32x2 ap, s, bp;\n\t"
      "sub.rn.f32x2 t1, a, ap;\n\t"
      "sub.rn.f32x2 t2, b, bp;\n\t"
      "add.rn.f32x2 e, t1, t2;\n\t"
      "shl.b32 cx, %2, 16;\n\t"
      "and.b32 cy, %2, 0xffff0000;\n\t"
      "mov.b64 c, {cx, cy};\n\t"
      "add.rn.f32x2 q, c, e;\n\t"
      "mov.b64 {q0, q1}, q;\n\t"
      "cvt.rn.bf16x2.f32 %2, q1, q0;\n\t"
      "mov.b64 {%0, %1}, s;\n\t"
      "}"
      : "+f"(a0), "+f"(a1), "+r"(r)
      : "r"(b0), "r"(b1));
  rl = *reinterpret_cast<const __nv_bfloat162*>(&r);
}

// Wait for one accumulation unit, fold its 32-lane x BN/4-column slice into
// the double-float running sum (rh + rl), and release the TMEM buffer.  The
// compensation rl (|rl| <~ 2^-24 |rh| per drain) is kept as packed bfloat16:
// rounding it to 8 bits costs ~2^-33 |rh| per drain, far below the target,
// and halves its register footprint.
template <int COLS>
__device__ __forceinline__ bool drain_unit(uint32_t taddr, uint64_t* full_bar, uint64_t* empty_bar, uint32_t parity,
                                           volatile int* abort_flag, uint64_t wait_ns, int lane,
                                           float (&rh)[COLS], __nv_bfloat162 (&rl)[COLS / 2]) {
  // the lanes agree before the warp-collective tensor-memory loads: a wait
  // that expired in any lane aborts the whole warp
  const bool got = ptx::mbar_wait_bounded(ptx::smem_u32(full_bar), parity, abort_flag, wait_ns);
  if (!__all_sync(0xffffffffu, got)) return false;
  ptx::tc_fence_after();
#pragma unroll
  for (int g = 0; g < COLS / 16; ++g) {
    uint32_t v[16];
    ptx::tmem_ld_32x32b_x16(taddr + g * 16, v);
    ptx::tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 16; j += 2)
      two_sum2_fold(rh[g * 16 + j], rh[g * 16 + j + 1], v[j], v[j + 1], rl[(g * 16 + j) / 2]);
  }
  ptx::tc_fence_before();
  if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(empty_bar));
  return true;
}

// GATE: grouped launches with gate-epilogue problems (out_mode 3)
template <bool G, int NPROD, bool DOTS, int BN, bool GATE = false>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_split_bf16_gemm(const __grid_constant__ GemmProblem single, const GemmParams p) {
  using TN = TileN<BN>;
  static_assert(BN == TBN || G, "narrow tiles are for grouped launches");
  static_assert(!(G && DOTS), "fused dot products are for single (non-grouped) FP64 problems");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TN::kStages * TN::kStageBytes);
  uint64_t* empty = full + TN::kStages;
  uint64_t* d1f = empty + TN::kStages;   // D1 buffer full (MMA -> epilogue)
  uint64_t* d1e = d1f + 2;          // D1 buffer empty (epilogue -> MMA)
  uint64_t* xf = d1e + 2;
  uint64_t* xe = xf + 2;
  uint64_t* done = xe + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  double* dacc = (double*)(smem + TN::kStages * TN::kStageBytes + 256);   // [NEPI][kMaxDots] per-warp dot sums
  if (DOTS)
    for (int i = threadIdx.x; i < NEPI * kMaxDots; i += blockDim.x) dacc[i] = 0.0;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TN::kStages; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_u32(&d1f[b]), 1);
      ptx::mbar_init(ptx::smem_u32(&d1e[b]), NEPI);
      ptx::mbar_init(ptx::smem_u32(&xf[b]), 1);
      ptx::mbar_init(ptx::smem_u32(&xe[b]), NEPI);
    }
    ptx::mbar_init(ptx::smem_u32(done), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (!G && warp == 0 && lane == 0) {
    ptx::tma_prefetch_desc(&single.tmA);
    ptx::tma_prefetch_desc(&single.tmB);
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), TN::kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int num_tiles = p.num_tiles;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued = 0, issued_phase = 0;   // bit s: stage s used / its last phase
      for (int tile = blockIdx.x; tile < num_tiles && !*abort_flag; tile += gridDim.x) {
        const GemmProblem* pr = find_problem<G>(tile, &single, p);
        const int lt = tile - pr->tile_begin;
        int mb, nb;
        tile_coords(lt, pr->num_m, pr->num_n, p.raster, mb, nb);
        const int nkb = pr->num_kb;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!ptx::mbar_wait_bounded(ptx::smem_u32(&empty[stage]), phase ^ 1, abort_flag, p.wait_ns)) break;
          const uint32_t fb = ptx::smem_u32(&full[stage]);
          ptx::mbar_arrive_expect_tx(fb, TN::kStageBytes);
          uint8_t* sa = smem + stage * TN::kStageBytes;
          ptx::tma_load_3d(ptx::smem_u32(sa), &pr->tmA, fb, kb * TBK, mb * TBM, 0);
          ptx::tma_load_3d(ptx::smem_u32(sa + STAGE_A), &pr->tmB, fb, kb * TBK, nb * BN, 0);
          issued |= 1u << stage;
          issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
          if (++stage == TN::kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // no copy may still be writing shared memory when the CTA exits
      for (int s = 0; s < TN::kStages; ++s) {
        if (!((issued >> s) & 1u)) continue;
        uint64_t t0 = ptx::globaltimer();
        while (!ptx::mbar_try_wait(ptx::smem_u32(&full[s]), (issued_phase >> s) & 1u))
          if (ptx::globaltimer() - t0 > WAIT_LIMIT_NS) break;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = ptx::idesc_bf16_f32(TBM, BN);
    // descriptors are built once; a stage, a piece or a 16-deep k-step only
    // adds a constant to the start-address field (address >> 4)
    const uint64_t desc0 = ptx::smem_desc_kmajor(ptx::smem_u32(smem), 64);
    constexpr uint64_t kStage = TN::kStageBytes >> 4, kB = STAGE_A >> 4, kPA = PIECE_A >> 4, kPB = TN::kPieceB >> 4;
    constexpr uint64_t kKs = 32 >> 4;
    int stage = 0;
    uint32_t u1 = 0, ux = 0;   // D1 / X accumulation-unit counters
    bool live = true;          // false after an abort: keep the barrier sequence, issue nothing
    bool grp_open = false;     // inside a k-block group the watcher handed over in one sync
    const int kb_d1 = p.kb_d1, kb_x = p.kb_x;   // in registers: the loop reads no memory
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
      if (live && *abort_flag) live = false;   // one shared-memory read per tile
      const int nkb = tile_kblocks<G>(tile, &single, p);
      uint32_t xbuf = 0;
      int c1 = 0, cx = 0;   // k-blocks into the current D1 / X accumulation unit
      for (int kb = 0; kb < nkb; ++kb) {
        const bool d1_first = c1 == 0;
        const bool x_first = cx == 0;
        const bool d1_last = c1 + 1 == kb_d1 || kb + 1 == nkb;
        const bool x_last = cx + 1 == kb_x || kb + 1 == nkb;
        c1 = d1_last ? 0 : c1 + 1;
        cx = x_last ? 0 : cx + 1;
        const uint32_t b1 = u1 & 1;
        if (x_first) xbuf = ux & 1;
        // the watcher saw this group's stages land (and, at unit starts, the buffers drained)
        if (!grp_open) named_bar_sync(kStageBar + stage, 64);   // once per group
        grp_open = (stage & 1) == 0 && kb + 1 < nkb;             // the group goes on past this k-block
        if (lane == 0 && !live) {
          ptx::mma_commit(ptx::smem_u32(&empty[stage]));   // the watcher's abort path waits on it
        } else if (lane == 0) {
          ptx::tc_fence_after();
          const uint64_t a = desc0 + (uint64_t)stage * kStage;
          const uint64_t b = a + kB;
          const uint32_t dD1 = tmem + b1 * BN;
          const uint32_t dX = tmem + 2 * BN + xbuf * BN;
          const uint32_t acc1 = d1_first ? 0u : 1u, accx = x_first ? 0u : 1u;
          // per 16-deep k-step: hi*hi into D1, cross products (A_i, B_j) with i + j in {1, 2}
          // into X, ordered by A piece so each A piece is read from shared memory once
#pragma unroll
          for (int ks = 0; ks < TBK / 16; ++ks) {
            const uint64_t ak = a + ks * kKs, bk = b + ks * kKs;
            const uint32_t f1 = ks ? 1u : acc1, fx = ks ? 1u : accx;
            if (NPROD == 6) {
              ptx::mma_f16_coll<ptx::kCollFill>(dD1, ak, bk, idesc, f1);                    // A0 B0
              ptx::mma_f16_coll<ptx::kCollUse>(dX, ak, bk + kPB, idesc, fx);                // A0 B1
              ptx::mma_f16_coll<ptx::kCollLastUse>(dX, ak, bk + 2 * kPB, idesc, 1u);        // A0 B2
              ptx::mma_f16_coll<ptx::kCollFill>(dX, ak + kPA, bk, idesc, 1u);               // A1 B0
              ptx::mma_f16_coll<ptx::kCollLastUse>(dX, ak + kPA, bk + kPB, idesc, 1u);      // A1 B1
              ptx::mma_f16(dX, ak + 2 * kPA, bk, idesc, 1u);                                // A2 B0
            } else {
              ptx::mma_f16_coll<ptx::kCollFill>(dD1, ak, bk, idesc, f1);                    // A0 B0
              ptx::mma_f16_coll<ptx::kCollLastUse>(dX, ak, bk + kPB, idesc, fx);            // A0 B1
              ptx::mma_f16(dX, ak + kPA, bk, idesc, 1u);                                    // A1 B0
            }
          }
          ptx::mma_commit(ptx::smem_u32(&empty[stage]));
          if (d1_last) ptx::mma_commit(ptx::smem_u32(&d1f[b1]));
          if (x_last) ptx::mma_commit(ptx::smem_u32(&xf[xbuf]));
        }
        if (d1_last) ++u1;
        if (x_last) ++ux;
        if (++stage == TN::kStages) stage = 0;
      }
    }
    if (lane == 0) {
      // all issued MMAs complete before TMEM is released
      ptx::mma_commit(ptx::smem_u32(done));
      uint64_t t0 = ptx::globaltimer();
      while (!ptx::mbar_try_wait(ptx::smem_u32(done), 0))
        if (ptx::globaltimer() - t0 > WAIT_LIMIT_NS) break;
    }
    __syncwarp();
  } else if (warp == kWatchWarp) {
    // ------------------------------------------------------------ watcher
    // Same tile / k-block / unit sequence as the MMA warp, run to its end: lane 0
    // waits (bounded) for each k-block's stage, and at a unit start for the
    // accumulator buffer it reuses; after the second k-block of a stage pair the
    // warp arrives on the pair's barrier.  After a failed wait (abort) it waits
    // only for the stage's previous commit before arriving (see the header).
    int stage = 0;
    uint32_t phase = 0;
    uint32_t u1 = 0, ux = 0;
    int use = 0;   // k-blocks seen so far (use of the current stage = use / TN::kStages)
    bool w_open = false;   // inside a group (its barrier is named by its first stage, grp_start)
    int grp_start = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
      const int nkb = tile_kblocks<G>(tile, &single, p);
      int c1 = 0, cx = 0;
      for (int kb = 0; kb < nkb; ++kb, ++use) {
        const bool d1_first = c1 == 0;
        const bool x_first = cx == 0;
        const bool d1_last = c1 + 1 == p.kb_d1 || kb + 1 == nkb;
        const bool x_last = cx + 1 == p.kb_x || kb + 1 == nkb;
        c1 = d1_last ? 0 : c1 + 1;
        cx = x_last ? 0 : cx + 1;
        if (lane == 0) {
          if (ok && d1_first)
            ok = ptx::mbar_wait_spin(ptx::smem_u32(&d1e[u1 & 1]), ((u1 >> 1) & 1) ^ 1, abort_flag, p.wait_ns);
          if (ok && x_first)
            ok = ptx::mbar_wait_spin(ptx::smem_u32(&xe[ux & 1]), ((ux >> 1) & 1) ^ 1, abort_flag, p.wait_ns);
          if (ok) ok = ptx::mbar_wait_spin(ptx::smem_u32(&full[stage]), phase, abort_flag, p.wait_ns);
          if (!ok && use >= TN::kStages) {
            // abort: arrive only once the MMA warp committed this stage's previous use
            // (it has passed that sync; the commit lands when the tensor cores finish)
            const uint64_t t0 = ptx::globaltimer();
            while (!ptx::mbar_test_wait(ptx::smem_u32(&empty[stage]), phase ^ 1))
              if (ptx::globaltimer() - t0 > WAIT_LIMIT_NS) break;
          }
        }
        __syncwarp();
        // one arrival per group, after its last k-block: an odd stage or the tile's last k-block
        if (!w_open) grp_start = stage;
        const bool grp_end = (stage & 1) == 1 || kb + 1 == nkb;
        if (grp_end) named_bar_arrive(kStageBar + grp_start, 64);
        w_open = !grp_end;
        if (d1_last) ++u1;
        if (x_last) ++ux;
        if (++stage == TN::kStages) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;                    // 0..NEPI-1
    const int qd = warp & 3;                    // TMEM lane quadrant of this warp
    const int c0 = (ew >> 2) * TN::kCols;   // first column of this warp
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    uint32_t u1 = 0, ux = 0;
    bool ok = true;
    float rh[TN::kCols];
    __nv_bfloat162 rl2[TN::kCols / 2];
    // Fused dot products: the tile this warp stored last is "pending"; its work
    // items (basis vector i, 16-column half h) run at the service points of the
    // next tile (after each accumulator drain), so the FP64 pipe works while the
    // tensor cores do; the last tile's items run after the loop.  Each item is
    // one warp-wide sum added to this warp's slot: a fixed order per CTA.
    int64_t d_off = 0;      // flat offset of this thread's 32 columns of the pending tile
    int d_cols = 0;         // valid columns among them (0: row outside the problem)
    int d_next = 0, d_items = 0;
    auto d_service = [&](int upto) {
      if (upto > d_items) upto = d_items;
      for (; d_next < upto; ++d_next) {
        const int i = d_next >> 1, h = d_next & 1;
        const double* wp = (const double*)single.C + d_off + h * 16;
        const double* vp = i < p.dot_nv ? p.dot_V + (int64_t)i * p.dot_ldv + d_off + h * 16 : wp;
        double acc = 0.0;
        if (d_cols >= h * 16 + 16) {
#pragma unroll
          for (int c = 0; c < 16; c += 2) {
            const double2 a = *(const double2*)(wp + c), b = *(const double2*)(vp + c);
            acc = fma(a.x, b.x, acc);
            acc = fma(a.y, b.y, acc);
          }
        } else {
          for (int c = 0; c < 16; ++c)
            if (h * 16 + c < d_cols) acc = fma(wp[c], vp[c], acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) dacc[ew * kMaxDots + i] += acc;
      }
    };
    // finish the pending tile, then make the tile just stored (row, first column) pending
    auto d_push = [&](int64_t row, int64_t n0, int64_t PM, int64_t PN, int64_t scm, int nkb) {
      d_service(d_items);
      d_off = row * scm + n0;
      d_cols = row < PM ? (int)max((int64_t)0, min((int64_t)TN::kCols, PN - n0)) : 0;
      d_next = 0;
      d_items = 2 * (p.dot_nv + 1);
      (void)nkb;
    };
    int d_quota = 1;        // items per service point while the next tile drains
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      const GemmProblem* pr = find_problem<G>(tile, &single, p);
      const int lt = tile - pr->tile_begin;
      int mb, nb;
        tile_coords(lt, pr->num_m, pr->num_n, p.raster, mb, nb);
      const int nkb = pr->num_kb;
      const int64_t PM = pr->M, PN = pr->N, scm = pr->scm, scn = pr->scn;
      void* const PC = pr->C;
      const int out_mode = pr->out_mode;
      if (nkb > 0 && nkb <= p.kb_d1 && nkb <= p.kb_x) {
        // One accumulation unit of each kind (short K, e.g. small sector blocks):
        // fold hi*hi and the cross products while storing, without the running
        // double-float sum.  FP64 output is the exact D1 + X, FP32 output its
        // single rounding, the pair output the error-free TwoSum pair.
        bool got = ptx::mbar_wait_bounded(ptx::smem_u32(&d1f[u1 & 1]), (u1 >> 1) & 1, abort_flag, p.wait_ns);
        if (got) got = ptx::mbar_wait_bounded(ptx::smem_u32(&xf[ux & 1]), (ux >> 1) & 1, abort_flag, p.wait_ns);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t td = tmem + lane_base + (u1 & 1) * BN + c0;
        const uint32_t tx = tmem + lane_base + 2 * BN + (ux & 1) * BN + c0;
        const int64_t row = (int64_t)mb * TBM + qd * 32 + lane;
        const int64_t n0 = (int64_t)nb * BN + c0;
#pragma unroll
        for (int g = 0; g < TN::kCols / 16; ++g) {
          uint32_t vd[16], vx[16];
          ptx::tmem_ld_32x32b_x16(td + g * 16, vd);
          ptx::tmem_ld_32x32b_x16(tx + g * 16, vx);
          ptx::tmem_ld_wait();
          if (GATE && out_mode == 3) {   // whole warp: the gate pairs rows of two lanes
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(vd[j]) + __uint_as_float(vx[j]);
            gate16(v, row, n0 + g * 16, pr, p);
            continue;
          }
          if (row >= PM) continue;
          const int64_t ng = n0 + g * 16;
          if (out_mode == 1) {
            float* crow = (float*)PC + row * scm;
            const bool vec = scn == 1 && ((((uintptr_t)(crow + ng)) & 15) == 0) && ng + 16 <= PN;
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const float4 o = make_float4(__uint_as_float(vd[j]) + __uint_as_float(vx[j]),
                                           __uint_as_float(vd[j + 1]) + __uint_as_float(vx[j + 1]),
                                           __uint_as_float(vd[j + 2]) + __uint_as_float(vx[j + 2]),
                                           __uint_as_float(vd[j + 3]) + __uint_as_float(vx[j + 3]));
              if (vec) {
                *(float4*)(crow + ng + j) = o;
              } else {
                if (ng + j < PN) crow[(ng + j) * scn] = o.x;
                if (ng + j + 1 < PN) crow[(ng + j + 1) * scn] = o.y;
                if (ng + j + 2 < PN) crow[(ng + j + 2) * scn] = o.z;
                if (ng + j + 3 < PN) crow[(ng + j + 3) * scn] = o.w;
              }
            }
          } else if (out_mode == 2) {
            float2* crow = (float2*)PC + row * scm;
            const bool vec = scn == 1 && ((((uintptr_t)(crow + ng)) & 15) == 0) && ng + 16 <= PN;
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
              float4 o;
              two_sum(__uint_as_float(vd[j]), __uint_as_float(vx[j]), o.x, o.y);
              two_sum(__uint_as_float(vd[j + 1]), __uint_as_float(vx[j + 1]), o.z, o.w);
              if (vec) {
                *(float4*)(crow + ng + j) = o;
              } else {
                if (ng + j < PN) crow[(ng + j) * scn] = make_float2(o.x, o.y);
                if (ng + j + 1 < PN) crow[(ng + j + 1) * scn] = make_float2(o.z, o.w);
              }
            }
          } else {
            double* crow = (double*)PC + row * scm;
            const bool vec = scn == 1 && ((((uintptr_t)(crow + ng)) & 15) == 0) && ng + 16 <= PN;
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
              const double2 o = make_double2((double)__uint_as_float(vd[j]) + (double)__uint_as_float(vx[j]),
                                             (double)__uint_as_float(vd[j + 1]) + (double)__uint_as_float(vx[j + 1]));
              if (vec) {
                *(double2*)(crow + ng + j) = o;
              } else {
                if (ng + j < PN) crow[(ng + j) * scn] = o.x;
                if (ng + j + 1 < PN) crow[(ng + j + 1) * scn] = o.y;
              }
            }
          }
        }
        ptx::tc_fence_before();
        if (lane == 0) {
          ptx::mbar_arrive(ptx::smem_u32(&d1e[u1 & 1]));
          ptx::mbar_arrive(ptx::smem_u32(&xe[ux & 1]));
        }
        ++u1;
        ++ux;
        if (DOTS) d_push(row, n0, PM, PN, scm, nkb);
        continue;
      }
#pragma unroll
      for (int j = 0; j < TN::kCols; ++j) rh[j] = 0.f;
#pragma unroll
      for (int j = 0; j < TN::kCols / 2; ++j) rl2[j] = __floats2bfloat162_rn(0.f, 0.f);
      int c1 = 0, cx = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const bool d1_last = c1 + 1 == p.kb_d1 || kb + 1 == nkb;
        const bool x_last = cx + 1 == p.kb_x || kb + 1 == nkb;
        c1 = d1_last ? 0 : c1 + 1;
        cx = x_last ? 0 : cx + 1;
        if (d1_last) {
          ok = drain_unit(tmem + lane_base + (u1 & 1) * BN + c0, &d1f[u1 & 1], &d1e[u1 & 1], (u1 >> 1) & 1,
                          abort_flag, p.wait_ns, lane, rh, rl2);
          ++u1;
          if (DOTS && ok) d_service(d_next + d_quota);
        }
        if (ok && x_last) {
          ok = drain_unit(tmem + lane_base + 2 * BN + (ux & 1) * BN + c0, &xf[ux & 1], &xe[ux & 1], (ux >> 1) & 1,
                          abort_flag, p.wait_ns, lane, rh, rl2);
          ++ux;
        }
        if (!ok) break;
      }
      if (!ok) break;
      // store the tile (one rounding of hi + lo)
      const int64_t row = (int64_t)mb * TBM + qd * 32 + lane;
      const int64_t n0 = (int64_t)nb * BN + c0;
      if (GATE && out_mode == 3) {   // gate epilogue (whole warp)
#pragma unroll
        for (int g = 0; g < TN::kCols / 16; ++g) {
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const float2 c = __bfloat1622float2(rl2[(g * 16 + j) / 2]);
            v[j] = rh[g * 16 + j] + c.x;
            v[j + 1] = rh[g * 16 + j + 1] + c.y;
          }
          gate16(v, row, n0 + g * 16, pr, p);
        }
      } else if (row < PM) {
        if (out_mode == 1) {
          float* crow = (float*)PC + row * scm;
          const bool vec = scn == 1 && ((((uintptr_t)(crow + n0)) & 15) == 0) && n0 + TN::kCols <= PN;
#pragma unroll
          for (int j = 0; j < TN::kCols; j += 4) {
            const float2 c01 = __bfloat1622float2(rl2[j / 2]);
            const float2 c23 = __bfloat1622float2(rl2[j / 2 + 1]);
            const float4 o = make_float4(rh[j] + c01.x, rh[j + 1] + c01.y, rh[j + 2] + c23.x, rh[j + 3] + c23.y);
            if (vec) {
              *(float4*)(crow + n0 + j) = o;
            } else {
              if (n0 + j < PN) crow[(n0 + j) * scn] = o.x;
              if (n0 + j + 1 < PN) crow[(n0 + j + 1) * scn] = o.y;
              if (n0 + j + 2 < PN) crow[(n0 + j + 2) * scn] = o.z;
              if (n0 + j + 3 < PN) crow[(n0 + j + 3) * scn] = o.w;
            }
          }
        } else if (out_mode == 2) {
          float2* crow = (float2*)PC + row * scm;
          const bool vec = scn == 1 && ((((uintptr_t)(crow + n0)) & 15) == 0) && n0 + TN::kCols <= PN;
#pragma unroll
          for (int j = 0; j < TN::kCols; j += 2) {
            const float2 c = __bfloat1622float2(rl2[j / 2]);
            float4 o;
            two_sum(rh[j], c.x, o.x, o.y);
            two_sum(rh[j + 1], c.y, o.z, o.w);
            if (vec) {
              *(float4*)(crow + n0 + j) = o;
            } else {
              if (n0 + j < PN) crow[(n0 + j) * scn] = make_float2(o.x, o.y);
              if (n0 + j + 1 < PN) crow[(n0 + j + 1) * scn] = make_float2(o.z, o.w);
            }
          }
        } else {
          double* crow = (double*)PC + row * scm;
          const bool vec = scn == 1 && ((((uintptr_t)(crow + n0)) & 15) == 0) && n0 + TN::kCols <= PN;
#pragma unroll
          for (int j = 0; j < TN::kCols; j += 2) {
            const float2 c = __bfloat1622float2(rl2[j / 2]);
            const double2 o = make_double2((double)rh[j] + (double)c.x, (double)rh[j + 1] + (double)c.y);
            if (vec) {
              *(double2*)(crow + n0 + j) = o;
            } else {
              if (n0 + j < PN) crow[(n0 + j) * scn] = o.x;
              if (n0 + j + 1 < PN) crow[(n0 + j + 1) * scn] = o.y;
            }
          }
        }
      }
      if (DOTS) {
        d_push(row, n0, PM, PN, scm, nkb);
        const int ndr = (nkb + p.kb_d1 - 1) / p.kb_d1;   // service points of the next tile (same K)
        d_quota = (d_items + ndr - 1) / ndr;
      }
    }
    if (DOTS) d_service(d_items);
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicExch(p.status, 1);
  if (DOTS && warp == 2) {
    // this CTA's partial sums, warps in order
    for (int i = lane; i <= p.dot_nv; i += 32) {
      double sum = 0.0;
      for (int e = 0; e < NEPI; ++e) sum += dacc[e * kMaxDots + i];
      p.dot_part[(int64_t)i * p.dot_stride + blockIdx.x] = sum;
    }
  }
  if (warp == 1) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, TN::kTmemCols);
  }
}

// ---------------------------------------------------------------- tensor maps
typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled_t get_encode_fn() {
  static PFN_encodeTiled_t fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_encodeTiled_t)ptr;
  }
  return fn;
}

}  // namespace

// 3-D map over bf16 piece planes [3][rows][Kp] with a {TBK, box_rows, 3} box;
// the planes are plane_rows * Kp elements apart (plane_rows >= rows; a row
// range of a larger piece matrix passes its own base and the full count).
tci_status tci_make_piece_map(tci_context ctx, CUtensorMap* map, const void* base, int64_t rows, int64_t Kp,
                              int box_rows, int64_t plane_rows) {
  PFN_encodeTiled_t enc = get_encode_fn();
  if (!enc) return tci_fail(ctx, TCI_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
  if (Kp % 8 != 0 || ((uintptr_t)base & 15)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "piece map: misaligned operand");
  if (plane_rows < rows) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "piece map: plane stride below the row count");
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, 3};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)(plane_rows * Kp * 2)};
  cuuint32_t box[3] = {(cuuint32_t)TBK, (cuuint32_t)box_rows, 3};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return tci_fail(ctx, TCI_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TCI_OK;
}

static tci_status fill_problem(tci_context ctx, GemmProblem* pr, int64_t M, int64_t N, int64_t Kp, const void* Ap,
                               const void* Bp, void* C, int out_mode, int64_t scm, int64_t scn,
                               int64_t a_plane_rows = 0, int64_t b_plane_rows = 0, int bn = TBN) {
  if (M <= 0 || N <= 0 || Kp <= 0) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split gemm: empty problem");
  if (M > (int64_t)INT32_MAX || N > (int64_t)INT32_MAX || Kp > (int64_t)INT32_MAX)
    return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "split gemm: dimension exceeds 2^31");
  memset(pr, 0, sizeof(*pr));
  TCI_TRY(tci_make_piece_map(ctx, &pr->tmA, Ap, M, Kp, TBM, a_plane_rows > 0 ? a_plane_rows : M));
  TCI_TRY(tci_make_piece_map(ctx, &pr->tmB, Bp, N, Kp, bn, b_plane_rows > 0 ? b_plane_rows : N));
  pr->C = C;
  pr->M = M;
  pr->N = N;
  pr->scm = scm;
  pr->scn = scn;
  pr->out_mode = out_mode;
  pr->num_m = (int)((M + TBM - 1) / TBM);
  pr->num_n = (int)((N + bn - 1) / bn);
  pr->num_kb = (int)((Kp + TBK - 1) / TBK);
  return TCI_OK;
}

static tci_status common_params(tci_context ctx, GemmParams* gp, int products, int chunk_k, int xchunk_k, int raster) {
  if (products != 6 && products != 3) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split gemm: products must be 3 or 6");
  static bool attr_set = false;
  if (!attr_set) {
    constexpr int S128 = TileN<128>::kSmem, S64 = TileN<64>::kSmem;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<false, 6, false, 128>, A, S128));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<true, 6, false, 128>, A, S128));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<false, 3, false, 128>, A, S128));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<true, 3, false, 128>, A, S128));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<false, 6, true, 128>, A, S128));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<false, 3, true, 128>, A, S128));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<true, 6, false, 64>, A, S64));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<true, 3, false, 64>, A, S64));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<true, 6, false, 128, true>, A, S128));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<true, 3, false, 128, true>, A, S128));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<true, 6, false, 64, true>, A, S64));
    TCI_CUDA(ctx, cudaFuncSetAttribute(k_split_bf16_gemm<true, 3, false, 64, true>, A, S64));
    attr_set = true;
  }
  gp->kb_d1 = chunk_k < TBK ? 1 : chunk_k / TBK;
  const int kx = xchunk_k < TBK ? 1 : xchunk_k / TBK;
  gp->kb_x = (kx + gp->kb_d1 - 1) / gp->kb_d1 * gp->kb_d1;   // X drains line up with D1 drains
  gp->products = products;
  gp->raster = raster;
  gp->status = ctx->d_status;
  gp->wait_ns = ctx->wait_limit_ns ? ctx->wait_limit_ns : WAIT_LIMIT_NS;
  return TCI_OK;
}

tci_status tci_gemm_split_bf16(tci_context ctx, int64_t M, int64_t N, int64_t Kp, const void* Ap, const void* Bp,
                               void* C, int out_mode, int64_t scm, int64_t scn, int products, int chunk_k,
                               int xchunk_k, int raster) {
  return tci_gemm_split_bf16_sub(ctx, M, N, Kp, Ap, M, Bp, N, C, out_mode, scm, scn, products, chunk_k, xchunk_k,
                                 raster);
}

tci_status tci_gemm_split_bf16_sub(tci_context ctx, int64_t M, int64_t N, int64_t Kp, const void* Ap,
                                   int64_t a_plane_rows, const void* Bp, int64_t b_plane_rows, void* C, int out_mode,
                                   int64_t scm, int64_t scn, int products, int chunk_k, int xchunk_k, int raster) {
  if (M <= 0 || N <= 0) return TCI_OK;
  if (out_mode < 0 || out_mode > 2) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split gemm: out_mode 0, 1 or 2");
  GemmProblem pr;
  TCI_TRY(fill_problem(ctx, &pr, M, N, Kp, Ap, Bp, C, out_mode, scm, scn, a_plane_rows, b_plane_rows));
  GemmParams gp;
  memset(&gp, 0, sizeof gp);
  TCI_TRY(common_params(ctx, &gp, products, chunk_k, xchunk_k, raster));
  gp.nprob = 1;
  gp.num_tiles = pr.num_m * pr.num_n;
  const int grid = gp.num_tiles < ctx->num_sms ? gp.num_tiles : ctx->num_sms;
  if (products == 6)
    k_split_bf16_gemm<false, 6, false, 128><<<grid, NTHREADS, TileN<128>::kSmem, ctx->stream>>>(pr, gp);
  else
    k_split_bf16_gemm<false, 3, false, 128><<<grid, NTHREADS, TileN<128>::kSmem, ctx->stream>>>(pr, gp);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

// The same GEMM (one problem, FP64 output C[m*N + n]) with the fused dot
// products of its output: part[i*part_stride + b] (b < *grid_out) receives CTA
// b's partial sum of <V_i, C> for i < nv and of <C, C> for i = nv.
tci_status tci_gemm_split_bf16_dots(tci_context ctx, int64_t M, int64_t N, int64_t Kp, const void* Ap, const void* Bp,
                                    double* C, int products, int chunk_k, int xchunk_k, int raster, const double* V,
                                    int64_t ldv, int nv, double* part, int part_stride, int* grid_out) {
  if (M <= 0 || N <= 0) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split gemm dots: empty problem");
  if (nv < 0 || nv + 1 > kMaxDots || !part || (nv > 0 && !V))
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split gemm dots: up to %d vectors", kMaxDots - 1);
  if ((N & 1) || (ldv & 1) || ((uintptr_t)C & 15) || ((uintptr_t)V & 15))
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split gemm dots: 16-byte aligned rows required");
  GemmProblem pr;
  TCI_TRY(fill_problem(ctx, &pr, M, N, Kp, Ap, Bp, C, 0, N, 1));
  GemmParams gp;
  memset(&gp, 0, sizeof gp);
  TCI_TRY(common_params(ctx, &gp, products, chunk_k, xchunk_k, raster));
  gp.nprob = 1;
  gp.num_tiles = pr.num_m * pr.num_n;
  gp.dot_V = V;
  gp.dot_ldv = ldv;
  gp.dot_nv = nv;
  gp.dot_stride = part_stride;
  gp.dot_part = part;
  const int grid = gp.num_tiles < ctx->num_sms ? gp.num_tiles : ctx->num_sms;
  if (grid > part_stride) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split gemm dots: partial-sum rows too short");
  if (products == 6)
    k_split_bf16_gemm<false, 6, true, 128><<<grid, NTHREADS, TileN<128>::kSmem, ctx->stream>>>(pr, gp);
  else
    k_split_bf16_gemm<false, 3, true, 128><<<grid, NTHREADS, TileN<128>::kSmem, ctx->stream>>>(pr, gp);
  TCI_CUDA(ctx, cudaGetLastError());
  if (grid_out) *grid_out = grid;
  return TCI_OK;
}

// Grouped launch: build the device table once (plan time), launch many times.
struct tci_split_group {
  GemmProblem* d_table = nullptr;
  int2* d_tile_map = nullptr;
  int bn = TBN;   // tile width of every problem of the group
  bool gated = false;   // has gate-epilogue problems (the launch needs their pointers)
  int nprob = 0;
  int num_tiles = 0;
  int64_t flops_tc = 0;
};

tci_status tci_split_group_create(tci_context ctx, int n, const tci_split_problem* probs, tci_split_group** out,
                                  int bn) {
  *out = nullptr;
  if (bn != 64 && bn != 128) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split group: tile width 64 or 128");
  bool gated = false;
  for (int i = 0; i < n; ++i) {
    const tci_split_problem& q = probs[i];
    if (q.out_mode < 0 || q.out_mode > 3) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split group: out_mode 0..3");
    if (q.out_mode == 3) {   // rows (a, t1), columns (b, t2, re/im)
      if (q.M != 2 * q.g_chi || q.N != 4 * q.g_chi || q.g_off < 0 || q.th_off < 0)
        return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split group: malformed gate problem %d", i);
      gated = true;
    }
  }
  std::vector<GemmProblem> host;
  host.reserve(n);
  std::vector<int> order;
  for (int i = 0; i < n; ++i)
    if (probs[i].M > 0 && probs[i].N > 0 && probs[i].Kp > 0) order.push_back(i);
  // longest K first (static round-robin then schedules the long tiles early)
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return probs[a].Kp > probs[b].Kp; });
  int tiles = 0;
  for (int i : order) {
    const tci_split_problem& q = probs[i];
    GemmProblem pr;
    TCI_TRY(fill_problem(ctx, &pr, q.M, q.N, q.Kp, q.Ap, q.Bp, q.C, q.out_mode, q.scm, q.scn, q.a_plane_rows,
                         q.b_plane_rows, bn));
    pr.g_chi = q.g_chi;
    pr.g_off = q.g_off;
    pr.th_off = q.th_off;
    pr.tile_begin = tiles;
    tiles += pr.num_m * pr.num_n;
    host.push_back(pr);
  }
  tci_split_group* g = new tci_split_group();
  g->bn = bn;
  g->gated = gated;
  g->nprob = (int)host.size();
  g->num_tiles = tiles;
  if (g->nprob > 0) {
    std::vector<int2> map;
    map.reserve(tiles);
    for (int i = 0; i < g->nprob; ++i)
      for (int t = 0; t < host[i].num_m * host[i].num_n; ++t) map.push_back(make_int2(i, host[i].num_kb));
    tci_status s = tci_dev_alloc(ctx, sizeof(GemmProblem) * host.size(), (void**)&g->d_table);
    if (s == TCI_OK) s = tci_dev_alloc(ctx, sizeof(int2) * map.size(), (void**)&g->d_tile_map);
    if (s != TCI_OK) {
      tci_dev_free(g->d_table);
      delete g;
      return s;
    }
    cudaError_t e = cudaMemcpyAsync(g->d_table, host.data(), sizeof(GemmProblem) * host.size(),
                                   cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->d_tile_map, map.data(), sizeof(int2) * map.size(), cudaMemcpyHostToDevice, ctx->stream);
    // (copies from pageable host memory have read their source when the call returns)
    if (e != cudaSuccess) {
      tci_dev_free(g->d_table);
      tci_dev_free(g->d_tile_map);
      delete g;
      return tci_cuda_fail(ctx, e, "split group table upload");
    }
  }
  *out = g;
  return TCI_OK;
}

void tci_split_group_destroy(tci_split_group* g) {
  if (!g) return;
  tci_dev_free(g->d_table);
  tci_dev_free(g->d_tile_map);
  delete g;
}

tci_status tci_split_group_launch(tci_context ctx, const tci_split_group* g, int products, int chunk_k, int xchunk_k,
                                  int raster, const void* const* gate_ptrs) {
  if (!g || g->nprob == 0) return TCI_OK;
  if (g->gated && !gate_ptrs) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "split group: gate pointers required");
  GemmParams gp;
  memset(&gp, 0, sizeof gp);
  TCI_TRY(common_params(ctx, &gp, products, chunk_k, xchunk_k, raster));
  gp.table = g->d_table;
  gp.tile_map = g->d_tile_map;
  gp.gate_ptrs = reinterpret_cast<const float2* const*>(gate_ptrs);
  gp.nprob = g->nprob;
  gp.num_tiles = g->num_tiles;
  GemmProblem dummy;
  memset(&dummy, 0, sizeof dummy);
  const int grid = gp.num_tiles < ctx->num_sms ? gp.num_tiles : ctx->num_sms;
  const int smem = g->bn == 64 ? TileN<64>::kSmem : TileN<128>::kSmem;
  if (g->gated) {
    if (products == 6)
      (g->bn == 64 ? k_split_bf16_gemm<true, 6, false, 64, true> : k_split_bf16_gemm<true, 6, false, 128, true>)
          <<<grid, NTHREADS, smem, ctx->stream>>>(dummy, gp);
    else
      (g->bn == 64 ? k_split_bf16_gemm<true, 3, false, 64, true> : k_split_bf16_gemm<true, 3, false, 128, true>)
          <<<grid, NTHREADS, smem, ctx->stream>>>(dummy, gp);
  } else if (products == 6) {
    (g->bn == 64 ? k_split_bf16_gemm<true, 6, false, 64> : k_split_bf16_gemm<true, 6, false, 128>)
        <<<grid, NTHREADS, smem, ctx->stream>>>(dummy, gp);
  } else {
    (g->bn == 64 ? k_split_bf16_gemm<true, 3, false, 64> : k_split_bf16_gemm<true, 3, false, 128>)
        <<<grid, NTHREADS, smem, ctx->stream>>>(dummy, gp);
  }
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

// ---------------------------------------------------------------- K0 split
namespace {

// hi + mid + lo == fl32(x) exactly (each residual is exact in FP32).
__device__ __forceinline__ void split3_f32(float xf, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(xf);
  float r1 = xf - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}

template <typename T>
__global__ void k_split3(const T* __restrict__ src, int64_t rows, int64_t K, int64_t sr, int64_t sk,
                         __nv_bfloat16* __restrict__ out, int64_t Kp, int64_t plane) {
  const int64_t total = rows * Kp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / Kp, k = i - r * Kp;
    __nv_bfloat16 h, m, l;
    if (k < K) {
      split3_f32((float)src[r * sr + k * sk], h, m, l);
    } else {
      h = m = l = __float2bfloat16_rn(0.f);
    }
    out[i] = h;
    out[plane + i] = m;
    out[2 * plane + i] = l;
  }
}

}  // namespace

tci_status tci_launch_split3(tci_context ctx, tci_dtype dt, const void* src, int64_t rows, int64_t K, int64_t sr,
                             int64_t sk, void* out, int64_t Kp, int64_t plane_rows) {
  int64_t total = rows * Kp;
  if (total == 0) return TCI_OK;
  const int64_t plane = (plane_rows > 0 ? plane_rows : rows) * Kp;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
  if (dt == TCI_F64)
    k_split3<double><<<(int)blocks, 256, 0, ctx->stream>>>((const double*)src, rows, K, sr, sk, (__nv_bfloat16*)out, Kp, plane);
  else if (dt == TCI_F32)
    k_split3<float><<<(int)blocks, 256, 0, ctx->stream>>>((const float*)src, rows, K, sr, sk, (__nv_bfloat16*)out, Kp, plane);
  else
    return tci_fail(ctx, TCI_ERR_DTYPE, "split3: real dtype required");
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

