// Lanczos ground-state solve of H_eff on the device (textbook: Golub &
// Van Loan Sec. 10.1; full re-orthogonalisation by classical Gram-Schmidt,
// repeated where the first projection cancelled (Daniel, Gragg, Kaufman &
// Stewart 1976) or in every step on request; Sturm-sequence bisection,
// Sec. 8.4, and inverse iteration for the tridiagonal eigenpair).
//
// One step j, with the basis V = [v_0 .. v_j] resident in HBM:
//   w = H v_j                                   (the matvec; its input was
//                                                prepared with v_j)
//   pass 1: h = V^T w, ||w||^2;  alpha_j = h_j   (one read of V and w; opt-in on
//                                                split-BF16 plans with FP64 vectors:
//                                                formed in the matvec's GEMM2
//                                                epilogue from the output tiles it
//                                                stores, per-CTA partials summed in
//                                                order; slower on B300)
//   DGKS test: ||w - V h||^2 = ||w||^2 - |h|^2 < ||w||^2 / 2 ?
//   taken:   pass 2: w -= V h, then h' = V^T w and ||w||^2  (fused: V read
//                    once, w read and written)
//            pass 3: w -= V h', then ||w||^2                (fused)
//   skipped: pass 2': w -= V h, then ||w||^2                (fused)
//   (all passes are launched; device gates make the unused ones exit)
//   beta_j = ||w||;  v_{j+1} = w / beta_j, written with the next matvec's
//   input (its bfloat16 pieces on a split-BF16 plan) in the same pass.
//
// Reduced-precision update terms (FP64 vectors only).  In a Lanczos step
// the pass-1 coefficients h_0 .. h_{j-2} and all second-pass coefficients h'
// are small: the recurrence leaves only alpha_j and beta_{j-1}, so they are
// of the order of the rounding error of w (FP64 matvec) or of the matvec
// error (split BF16, ~1e-7 ||w||).  A device test takes the 1-norm of the k
// coefficients of such terms:
//   <= 2^-32 ||w|| / (k + 8): the terms are summed in FP32 from the basis
//      truncated to 24 significant bits (f32_trunc) and subtracted from w
//      with one FP64 FMA;
//   <= 2^-10 ||w|| / (k + 8), k >= 6 (fewer cost more than their FP64
//      FMAs): they are summed in double-float arithmetic (basis and
//      coefficients split into FP32 pairs, products made exact with FMA,
//      Dekker / Knuth sums);
// either way the error added is below 2^-56 ||w||, under the FP64 rounding
// of the update itself; otherwise the terms stay FP64.  The update pass is one
// launch whose blocks read the device's choice and run that arithmetic's
// body (each body compiled once per term arithmetic).  The second pass's h' are rounding-level after the
// first projection, so pass 3 is folded into the next-vector kernel (FP32
// terms), with beta_j^2 = ||w'||^2 - |h'|^2 (Pythagoras: w' - V h' is
// orthogonal to V up to rounding, and |h'| <= 2^-32 ||w'||).  The reduced
// terms only spare the FP64 pipe (B300 issues FP64 FMAs at ~1/64 of its FP32
// rate).
//
// Dot products.  FP64 (the default).  Opt-in on split plans with FP64 vectors
// (whose matvec error, ~1e-7 ||w||, dwarfs any rounding of the projections):
// the first projection's dots <v_i, w> and ||w||^2 summed in double-float
// arithmetic from a double-float shadow of the basis (each v_i also stored
// as an FP32 pair within 2^-47 |v_i|, written with v_i), and the second
// projection's dots from FP32 pairs split on the integer pipes in the
// double-float-terms update pass: both passes then run on the FP32 pipes and
// are bound by HBM, not by the FP64 rate.  Their error is ~2^-46 ||v_i||
// ||w||, above FP64 rounding; the recurrence scalars alpha, beta and every
// update stay FP64.
//
// Pass 1's update contains the three-term recurrence (h_j = alpha_j, h_{j-1}
// = beta_{j-1} up to rounding), so the step equals the three-term step
// followed by one or two classical Gram-Schmidt passes.  Without
// re-orthogonalisation: pass 1 takes only alpha_j and the last pass
// subtracts alpha_j v_j + beta_{j-1} v_{j-1}.
//
// Vector arithmetic (a policy template over the same kernels):
//   FP64          FP64 vectors, every dot product in FP64 (the default;
//                 small update terms reduced as above);
//   double-float  vectors held as FP32 pairs hi + lo (~48 significant bits)
//                 with error-free transformations, so the passes run on the
//                 FP32 pipes: B300 issues FP64 FMAs at ~1/64 of its FP32
//                 rate, which makes the FP64 passes FP64-pipe bound.
//
// All scalars (alpha, beta, Gram-Schmidt coefficients, stop flag, step
// count, Ritz coefficients) stay in device memory as FP64; the host enqueues
// the whole solve and reads back once at the end.  Reductions are
// deterministic: a fixed grid, a fixed per-thread order and an in-order sum
// of the block partials.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <map>
#include <mutex>
#include <type_traits>

#include "heff_plan.cuh"

namespace {

constexpr int NT = 256;
constexpr int NBMAX = 1184;      // partial-sum slots per vector (>= any pass's grid: one wave, <= 8 x 148)
constexpr int MAXM = 256;
constexpr int GMAX = 20;         // basis vectors per fused pass
// device scalar layout (doubles)
constexpr int OFF_ALPHA = 0;
constexpr int OFF_BETA = MAXM;
constexpr int OFF_H = 2 * MAXM;          // MAXM + 1 entries: pass-1 coefficients
constexpr int OFF_CTRL = 3 * MAXM + 8;   // [0] stop flag, [1] steps done, [2] theta, [3] sum of squares,
                                         // [4] pass-1 sum of squares, [5] [6] pass gates, [7] second passes
constexpr int OFF_Y = 3 * MAXM + 16;     // Ritz coefficients
constexpr int OFF_H2 = 4 * MAXM + 32;    // MAXM + 1 entries: pass-2 coefficients
constexpr int OFF_LO = 5 * MAXM + 40;    // FP32 rounding-level terms (LO_* below)
constexpr int NSCAL = 5 * MAXM + 64;
constexpr int OFF_TICKET = NSCAL - 4;    // blocks done in the current pass (as an unsigned; zero between passes)
// OFF_LO + : pass-2 / 2' FP32 terms (count, scale, inverse scale), pass-2
// ||w'||^2, pass-3 FP32 scale and inverse, gates (run while 0) of the FP32
// next-vector kernel, the FP64 pass 3 and the plain next-vector kernel,
// counters of FP32-term passes and fused pass-3 corrections.
constexpr int LO_NS1 = 0, LO_SC1 = 1, LO_ISC1 = 2, LO_WN2 = 3, LO_SC3 = 4, LO_ISC3 = 5;
constexpr int LO_GFAST = 6, LO_GSLOW = 7, LO_GNEXT = 8, LO_N1 = 9, LO_N3 = 10, LO_MODE1 = 11, LO_N2 = 12;
static_assert(OFF_LO + LO_N2 < OFF_TICKET, "scalar layout");
// Terms are summed in FP32 where their coefficients' 1-norm times (k + 8),
// k the number of such terms, is at most 2^-32 times the norm of the vector
// they update, and in double-float where it is at most 2^-10 times it.
constexpr double kF32Bound = 2.3283064365386963e-10;   // 2^-32
constexpr double kDFBound = 9.765625e-4;                // 2^-10
constexpr int kTermsF64 = 0, kTermsF32 = 1, kTermsDF = 2;
// the double-float-terms update whose dots are double-float too (opt-in, split
// plans): runs where the device chose kTermsDF
constexpr int kTermsDFDots = 3;
constexpr int64_t kReducedMinN = 1 << 20;               // vector length from which reduced terms are used
constexpr int kFusedMax = 23;                           // basis vectors whose dots the split GEMM can fuse

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// x truncated to an FP32 number with 24 significant bits, from the IEEE-754
// bit fields on the integer pipes (no FP64 instruction): the exponent is
// re-biased (1023 -> 127) and the top 23 fraction bits kept.  Exponents are
// clamped to FP32's normal range, so |x| < 2^-126 becomes a number of that
// size with x's sign (an absolute error below 2^-125) and |x| >= 2^128 the
// largest binade; NaN and infinity are not preserved (only basis vectors,
// |x| <= 1, come here).
// FP32 -> FP64 on the integer pipes for normal numbers and zero (the exact
// conversion: exponent rebiased by 896, fraction shifted by 29); subnormals,
// infinities and NaN take the conversion instruction (FP64 pipe).
__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned b = __float_as_uint(f), e = (b >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0u && (b & 0x7fffffu) == 0u) return __longlong_as_double((long long)sign);
  if (e == 0u || e == 0xffu) return (double)f;
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  unsigned a = min(max(hi & 0x7fffffffu, 0x38100000u), 0x47efffffu);   // exponent in [897, 1150]
  a -= 0x38000000u;                                                      // 1023 - 127 = 896
  return __uint_as_float(__funnelshift_l(lo, a, 3) | (hi & 0x80000000u));
}

// x = h + l to ~2^-47 |x| for 2^-126 <= |x| < 2^128: h = f32_trunc(x), l the
// 29 fraction bits below h's (their value m 2^(e - 1075), e the biased FP64
// exponent) rounded to FP32, with x's sign; l is 0 where that value is
// below FP32's normal range.
__device__ __forceinline__ void f32_split2(double x, float& h, float& l) {
  h = f32_trunc(x);
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int se = (int)((hi >> 20) & 0x7ffu) - 948;   // FP32 biased exponent of 2^(e - 1075)
  const float scale = se > 0 ? __uint_as_float((unsigned)se << 23) : 0.f;
  const float mag = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), scale);
  l = __uint_as_float(__float_as_uint(mag) | (hi & 0x80000000u));
}

// Shadow element of a basis value y: the FP32 pair of f32_split2 (integer
// pipes; no FP64 instruction), hi + lo within 2^-47 |y| (|y| <= 1).
__device__ __forceinline__ float2 shadow_of(double y) {
  float h, l;
  f32_split2(y, h, l);
  return make_float2(h, l);
}

// ---------------------------------------------------------------- double-float
// A double-float number is the unevaluated sum hi + lo of two FP32 values
// with |lo| <= ulp(hi)/2 (Dekker, Numer. Math. 18, 1971).  Sums use Knuth's
// TwoSum (TAOCP vol. 2, Sec. 4.2.2) and products the FMA-exact split
// a*b = p + e; running sums keep an unnormalised low word.

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ float2 df_norm(float h, float l) {
  float s, e;
  df_two_sum(h, l, s, e);
  return make_float2(s, e);
}

__device__ __forceinline__ float2 df_from_double(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// x * y as (p, t) with p + t = x*y to ~2^-48 relative
__device__ __forceinline__ void df_prod(float2 x, float2 y, float& p, float& t) {
  p = __fmul_rn(x.x, y.x);
  const float e = __fmaf_rn(x.x, y.x, -p);
  t = __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, e));
}

// ---------------------------------------------------------------- arithmetic policies
struct ArithF64 {
  using V = double;
  struct Acc { double s; };
  struct Coef { double c; };
  struct Sub { double w, s; };
  __device__ static Acc zero() { return {0.0}; }
  __device__ static void acc(Acc& a, V x, V y) { a.s = fma(x, y, a.s); }
  __device__ static void acc_c(Acc& a, Coef c, V y) { a.s = fma(c.c, y, a.s); }
  __device__ static double value(const Acc& a) { return a.s; }
  __device__ static double lane_total(const Acc& a) { return warp_sum(a.s); }   // valid in lane 0
  __device__ static Coef coef(double c) { return {c}; }
  __device__ static Sub sub_begin(V w) { return {w, 0.0}; }
  __device__ static void sub(Sub& t, Coef c, V v) { t.s = fma(c.c, v, t.s); }
  __device__ static V sub_end(const Sub& t) { return t.w - t.s; }
  __device__ static V mul(V x, Coef c) { return x * c.c; }
  __device__ static V from_double(double x) { return x; }
  __device__ static double to_double(V v) { return v; }
  __device__ static float f32(V v) { return __double2float_rn(v); }
};

struct ArithDF {
  using V = float2;
  struct Acc { float h, l; };
  struct Coef { float2 c; };
  struct Sub { float h, l; };
  __device__ static Acc zero() { return {0.f, 0.f}; }
  __device__ static void acc(Acc& a, V x, V y) {
    float p, t, s, e;
    df_prod(x, y, p, t);
    df_two_sum(a.h, p, s, e);
    a.h = s;
    a.l = __fadd_rn(a.l, __fadd_rn(e, t));
  }
  __device__ static void acc_c(Acc& a, Coef c, V y) { acc(a, c.c, y); }
  __device__ static double value(const Acc& a) { return (double)a.h + (double)a.l; }
  __device__ static double lane_total(const Acc& a) {   // double-float tree, one FP64 add at the end
    float h = a.h, l = a.l;
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
      float s, e;
      df_two_sum(h, h2, s, e);
      h = s;
      l = __fadd_rn(l, __fadd_rn(l2, e));
    }
    return (double)h + (double)l;
  }
  __device__ static Coef coef(double c) { return {df_from_double(c)}; }
  __device__ static Sub sub_begin(V w) { return {w.x, w.y}; }
  __device__ static void sub(Sub& t, Coef c, V v) {
    float p, q, s, e;
    df_prod(c.c, v, p, q);
    df_two_sum(t.h, -p, s, e);
    t.h = s;
    t.l = __fadd_rn(t.l, __fsub_rn(e, q));
  }
  __device__ static V sub_end(const Sub& t) { return df_norm(t.h, t.l); }
  __device__ static V mul(V x, Coef c) {
    float p, t;
    df_prod(x, c.c, p, t);
    return df_norm(p, t);
  }
  __device__ static V from_double(double x) { return df_from_double(x); }
  __device__ static double to_double(V v) { return (double)v.x + (double)v.y; }
  __device__ static float f32(V v) { return v.x; }   // fl32(hi + lo) = hi for a normalised pair
};

// ---------------------------------------------------------------- vector kernels
// Where a pass's last block puts the totals of its partial sums (dots: one per
// row, sq: the sum of squares); ticket null: the partials are left for
// k_reduce_parts.
struct PassOut {
  double* dots = nullptr;
  double* sq = nullptr;
  unsigned* ticket = nullptr;
};

// Per-block partial sums of G accumulators (fixed order): part[g*NBMAX +
// blockIdx.x] for g < nv.
// Called by every thread of the block; two calls with the same G in one
// kernel share `sh`, hence the barrier before it is written.
template <class A, int G>
__device__ __forceinline__ void block_partials(const typename A::Acc (&a)[G], int nv, double* part) {
  __shared__ double sh[NT / 32][G];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (g < nv) {
      const double s = A::lane_total(a[g]);
      if (lane == 0) sh[wid][g] = s;
    }
  __syncthreads();
  if (threadIdx.x < G && threadIdx.x < nv) {
    double s = 0.0;
    for (int k = 0; k < NT / 32; ++k) s += sh[k][threadIdx.x];
    part[(int64_t)threadIdx.x * NBMAX + blockIdx.x] = s;
  }
}

// With po.ticket: after every block has written its partials, the last block
// to finish (counted on the ticket) forms the totals the separate
// k_reduce_parts launches would, in the same order (so the same values): each
// of its 256 threads sums the slots b = t, t + 256, ... of every row, the
// rows' loads issued together, then each row goes through the same warp
// shuffle tree and the eight warp sums are added in order.  The ticket is
// cleared for the next pass.  Called by every thread of every block that
// wrote partials (nrows <= G rows NBMAX apart from part; part_sq: the
// sum-of-squares row).
template <int G>
__device__ __forceinline__ void pass_finish(const double* part, int nrows, const double* part_sq, const PassOut& po) {
  static_assert(NT == 256, "the totals follow k_reduce_parts' 256-thread order");
  if (!po.ticket) return;
  __shared__ int last;
  __shared__ double sh[NT / 32][G + 1];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(po.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int nb = gridDim.x, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nr = po.dots ? nrows : 0;
  double t[G + 1];
#pragma unroll
  for (int r = 0; r <= G; ++r) t[r] = 0.0;
  for (int b = threadIdx.x; b < nb; b += NT) {
#pragma unroll
    for (int r = 0; r < G; ++r)
      if (r < nr) t[r] += __ldcg(part + (int64_t)r * NBMAX + b);
    if (po.sq) t[G] += __ldcg(part_sq + b);
  }
#pragma unroll
  for (int r = 0; r <= G; ++r) {
    if (r < G && r >= nr) continue;
    if (r == G && !po.sq) continue;
    const double v = warp_sum(t[r]);
    if (lane == 0) sh[wid][r] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < nr || (po.sq && threadIdx.x == G)) {
    double v = 0.0;
    for (int k = 0; k < NT / 32; ++k) v += sh[k][threadIdx.x];
    if ((int)threadIdx.x < nr) po.dots[threadIdx.x] = v;
    else *po.sq = v;
  }
  if (threadIdx.x == 0) *po.ticket = 0u;
}

// partials of <V_{v0+g}, w>, g < nv <= G, into part rows v0 + g; with SQ
// also the partials of ||w||^2 into part_sq
template <class A, int G, bool SQ>
__global__ void __launch_bounds__(NT) k_dots(const typename A::V* __restrict__ V, int64_t ldv, int v0, int nv,
                                             const typename A::V* __restrict__ w, int64_t n, double* __restrict__ part,
                                             double* __restrict__ part_sq, const double* __restrict__ ctrl,
                                             const PassOut po) {
  if (ctrl[0] != 0.0) return;
  typename A::Acc a[G];
#pragma unroll
  for (int g = 0; g < G; ++g) a[g] = A::zero();
  typename A::Acc q = A::zero();
  using Vt = typename A::V;
  const Vt* Vb = V + (int64_t)v0 * ldv;
  int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * NT;
  if constexpr (std::is_same<A, ArithF64>::value) {
    // FP64 passes run with G == nv: two elements per iteration, every load
    // issued before the FMAs that use it (the same per-thread order of terms)
    if (nv == G) {
      for (; i + st < n; i += 2 * st) {
        const double x0 = w[i], x1 = w[i + st];
        double y0[G], y1[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          y0[g] = Vb[(int64_t)g * ldv + i];
          y1[g] = Vb[(int64_t)g * ldv + i + st];
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          A::acc(a[g], y0[g], x0);
          A::acc(a[g], y1[g], x1);
        }
        if (SQ) {
          A::acc(q, x0, x0);
          A::acc(q, x1, x1);
        }
      }
    }
  }
  for (; i < n; i += st) {
    const Vt x = w[i];
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < nv) A::acc(a[g], Vb[(int64_t)g * ldv + i], x);
    if (SQ) A::acc(q, x, x);
  }
  block_partials<A, G>(a, nv, part + (int64_t)v0 * NBMAX);
  if (SQ) {
    const typename A::Acc qa[1] = {q};
    block_partials<A, 1>(qa, 1, part_sq);
  }
  pass_finish<G>(part + (int64_t)v0 * NBMAX, nv, part_sq, po);
}

// Pass 1 from the double-float shadow of the basis (FP64 vectors; vector g's hi
// plane at Vs + 2 g ldv, its lo plane ldv after it): partials of
// <Vs_g, w>, g < nv <= G, into part rows g, and with SQ of ||w||^2; w (FP64) is
// split into an FP32 pair once per element on the integer pipes (f32_split2,
// within 2^-47 |w_i| where |w_i| >= 2^-126) and every product and sum runs in
// double-float arithmetic on the FP32 pipes: no FP64 instruction per element.
template <int G, bool SQ>
__global__ void __launch_bounds__(NT, 2) k_dots_shadow(const float* __restrict__ Vs, int64_t ldv, int nv,
                                                    const double* __restrict__ w, int64_t n,
                                                    double* __restrict__ part, double* __restrict__ part_sq,
                                                    const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  ArithDF::Acc a[G];
#pragma unroll
  for (int g = 0; g < G; ++g) a[g] = ArithDF::zero();
  ArithDF::Acc q = ArithDF::zero();
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
    // every load first (all in flight together), then the arithmetic; rows
    // g >= nv hold zeros and add nothing
    float2 vv[G];
#pragma unroll
    for (int g = 0; g < G; ++g)
      vv[g] = g < nv ? make_float2(__ldg(&Vs[2 * g * ldv + i]), __ldg(&Vs[(2 * g + 1) * ldv + i]))
                     : make_float2(0.f, 0.f);
    const float2 x = shadow_of(__ldg(&w[i]));
#pragma unroll
    for (int g = 0; g < G; ++g) ArithDF::acc(a[g], vv[g], x);
    if (SQ) ArithDF::acc(q, x, x);
  }
  block_partials<ArithDF, G>(a, nv, part);
  if (SQ) {
    const ArithDF::Acc qa[1] = {q};
    block_partials<ArithDF, 1>(qa, 1, part_sq);
  }
}

// w -= sum_{g<nv} coef[v0+g] V_{v0+g}; then (DOTS) partials of <V_{v0+g}, w>
// into part rows v0 + g and (SUMSQ) partials of ||w||^2 into part_sq.  In the
// kTermsDFDots variant (double-float terms; opt-in on split plans, whose
// update coefficients are at the matvec-error level) the dots also run in
// double-float arithmetic on the FP32 pipes, from the FP32 pairs of f32_split2
// (integer pipes) of both operands, so the pass stays HBM-bound; ||w||^2 stays
// FP64.  TERMS
// (FP64 vectors; v0 = 0, nv = G): the arithmetic of the first nv - 2 terms,
// kTermsF64, kTermsF32 or kTermsDF with coefficients scaled by lo[LO_SC1]
// (see the header); with lo the body runs only when it is the variant the
// device chose (lo[LO_MODE1] where lo[LO_NS1] = nv - 2, else kTermsF64).
template <class A, int G, bool DOTS, bool SUMSQ, int TERMS>
__device__ __forceinline__ void update_body(const typename A::V* __restrict__ V, int64_t ldv, int v0, int nv,
                                            const double* __restrict__ coef, typename A::V* __restrict__ w,
                                            int64_t n, double* __restrict__ part, double* __restrict__ part_sq,
                                            const double* __restrict__ ctrl, const double* __restrict__ lo,
                                            const PassOut& po) {
  using Vt = typename A::V;
  constexpr bool kF64 = std::is_same<Vt, double>::value;
  static_assert(kF64 || TERMS == kTermsF64, "reduced-precision terms need FP64 vectors");
  if (ctrl[0] != 0.0) return;
  if (kF64 && nv != G) {   // FP64 passes are dispatched with G == nv; anything else poisons w
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
      w[i] = A::from_double(__longlong_as_double(0x7ff8000000000000ll));
    return;
  }
  constexpr int kArith = TERMS == kTermsDFDots ? kTermsDF : TERMS;   // the term arithmetic
  if constexpr (kF64) {
    int mode = kTermsF64;
    if (lo && nv == G && nv > 2 && (int)lo[LO_NS1] == nv - 2) mode = (int)lo[LO_MODE1];
    if (mode != kArith) return;
  }
  __shared__ typename A::Coef cs[G];
  __shared__ float csf[G], csl[G];
  if (threadIdx.x < G) {
    const double c = threadIdx.x < nv ? coef[v0 + threadIdx.x] : 0.0;
    cs[threadIdx.x] = A::coef(c);
    if constexpr (TERMS != kTermsF64) {
      const double cc = c * lo[LO_SC1];   // exact: a power-of-two scale
      const float ch = (float)cc;
      csf[threadIdx.x] = ch;
      csl[threadIdx.x] = (float)(cc - (double)ch);
    }
  }
  double isc = 0.0;
  if constexpr (TERMS != kTermsF64) isc = lo[LO_ISC1];
  __syncthreads();
  constexpr int GD = DOTS ? G : 1;
  constexpr bool kDFDots = kF64 && DOTS && TERMS == kTermsDFDots;
  using DA = typename std::conditional<kDFDots, ArithDF, A>::type;
  typename DA::Acc d[GD];
#pragma unroll
  for (int g = 0; g < GD; ++g) d[g] = DA::zero();
  typename A::Acc q = A::zero();
  const Vt* Vb = V + (int64_t)v0 * ldv;
  const int64_t stride = (int64_t)gridDim.x * NT;
  int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x;
  // double-float vectors: software pipeline (the next element's loads are
  // issued before this element's arithmetic); FP64 vectors: a plain loop,
  // whose lower register count keeps more blocks resident to hide latency
  // (pipelined, the DGKS pass measured 5.27 -> 5.35 ms per chi = 2048 solve)
  constexpr bool kPipe = !kF64;
  Vt vn[kPipe ? G : 1], xn = Vt();
  if constexpr (kPipe) {
    if (i < n) {
      xn = w[i];
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < nv) vn[g] = Vb[(int64_t)g * ldv + i];
    }
  }
  for (; i < n; i += stride) {
    Vt v[G];
    Vt x;
    if constexpr (kPipe) {
#pragma unroll
      for (int g = 0; g < G; ++g) v[g] = vn[g];
      x = xn;
      if (i + stride < n) {
        xn = w[i + stride];
#pragma unroll
        for (int g = 0; g < G; ++g)
          if (g < nv) vn[g] = Vb[(int64_t)g * ldv + i + stride];
      }
    } else {
      // FP64 passes are launched with G == nv (exact-size instantiations)
#pragma unroll
      for (int g = 0; g < G; ++g) v[g] = Vb[(int64_t)g * ldv + i];
      x = w[i];
    }
    typename A::Sub t = A::sub_begin(x);
    Vt y;
    // the split point is fixed at compile time (terms 0 .. G-3 reduced, the
    // last two FP64): with a run-time bound the compiler would evaluate both
    // arithmetics for every term and select
    if constexpr (kArith == kTermsDF) {
      // double-float sum (sh + sl): c v = ch vh + (ch vl + cl vh) with ch vh
      // split exactly by FMA, the leading parts added by TwoSum
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int g = 0; g < G - 2; ++g) {
        float vh, vl;
        f32_split2(v[g], vh, vl);
        const float p = __fmul_rn(csf[g], vh);
        const float q = __fmaf_rn(csf[g], vl, __fmaf_rn(csl[g], vh, __fmaf_rn(csf[g], vh, -p)));
        float s2, e2;
        df_two_sum(sh, p, s2, e2);
        sh = s2;
        sl = __fadd_rn(sl, __fadd_rn(e2, q));
      }
#pragma unroll
      for (int g = G - 2 > 0 ? G - 2 : 0; g < G; ++g) A::sub(t, cs[g], v[g]);
      y = A::sub_end(t);
      // with dots the pass is bound by the FP64 pipe: its conversions run on the integer pipes
      if constexpr (DOTS)
        y = fma(-(f64_of_f32(sh) + f64_of_f32(sl)), isc, y);
      else
        y = fma(-((double)sh + (double)sl), isc, y);
    } else if constexpr (kArith == kTermsF32) {
      float sf = 0.f;
#pragma unroll
      for (int g = 0; g < G - 2; ++g) sf = __fmaf_rn(csf[g], f32_trunc(v[g]), sf);
#pragma unroll
      for (int g = G - 2 > 0 ? G - 2 : 0; g < G; ++g) A::sub(t, cs[g], v[g]);
      y = A::sub_end(t);
      y = fma(-(double)sf, isc, y);
    } else if constexpr (kF64) {
#pragma unroll
      for (int g = 0; g < G; ++g) A::sub(t, cs[g], v[g]);
      y = A::sub_end(t);
    } else {
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < nv) A::sub(t, cs[g], v[g]);
      y = A::sub_end(t);
    }
    w[i] = y;
    if constexpr (kDFDots) {
      const float2 yy = shadow_of(y);
#pragma unroll
      for (int g = 0; g < GD; ++g) ArithDF::acc(d[g], shadow_of(v[g]), yy);
    } else if (DOTS) {
#pragma unroll
      for (int g = 0; g < GD; ++g)
        if (kF64 || g < nv) A::acc(d[g], v[g], y);
    }
    if (SUMSQ) A::acc(q, y, y);
  }
  if (DOTS) block_partials<DA, GD>(d, nv, part + (int64_t)v0 * NBMAX);
  if (SUMSQ) {
    const typename A::Acc qa[1] = {q};
    block_partials<A, 1>(qa, 1, part_sq);
  }
  if (DOTS || SUMSQ) pass_finish<G>(part + (int64_t)v0 * NBMAX, DOTS ? nv : 0, part_sq, po);
}

template <class A, int G, bool DOTS, bool SUMSQ, int TERMS>
__global__ void __launch_bounds__(NT, (std::is_same<typename A::V, double>::value ? 2 : 1))
    k_update(const typename A::V* __restrict__ V, int64_t ldv, int v0, int nv, const double* __restrict__ coef,
             typename A::V* __restrict__ w, int64_t n, double* __restrict__ part, double* __restrict__ part_sq,
             const double* __restrict__ ctrl, const double* __restrict__ lo, const PassOut po) {
  update_body<A, G, DOTS, SUMSQ, TERMS>(V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
}

// One launch for an FP64 update pass whose term arithmetic the device chooses
// (lo given): the block reads the choice and runs that variant's body (the
// choice is uniform over the grid), instead of three launches of which two
// exit at once.  DFD: the double-float-terms variant forms its dots in
// double-float (kTermsDFDots).
// (Two blocks per SM: the DGKS variants of the largest bases spill a few
// registers there, and measured faster so than with one block's registers.)
template <int G, bool DOTS, bool SUMSQ, bool DFD>
__global__ void __launch_bounds__(NT, 2)
    k_update_sel(const double* __restrict__ V, int64_t ldv, int v0, int nv, const double* __restrict__ coef,
                 double* __restrict__ w, int64_t n, double* __restrict__ part, double* __restrict__ part_sq,
                 const double* __restrict__ ctrl, const double* __restrict__ lo, const PassOut po) {
  int mode = kTermsF64;
  if (nv == G && nv > 2 && (int)lo[LO_NS1] == nv - 2) mode = (int)lo[LO_MODE1];
  if (mode == kTermsF32)
    update_body<ArithF64, G, DOTS, SUMSQ, kTermsF32>(V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
  else if (mode == kTermsDF)
    update_body<ArithF64, G, DOTS, SUMSQ, (DOTS && DFD) ? kTermsDFDots : kTermsDF>(V, ldv, v0, nv, coef, w, n, part,
                                                                                 part_sq, ctrl, lo, po);
  else
    update_body<ArithF64, G, DOTS, SUMSQ, kTermsF64>(V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
}

__device__ __forceinline__ void split3_store(__nv_bfloat16* o, int64_t plane, float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const float r1 = __fsub_rn(x, __bfloat162float(h));
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const __nv_bfloat16 l = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(m)));
  o[0] = h;
  o[plane] = m;
  o[2 * plane] = l;
}

// Two consecutive elements (o 4-byte aligned): one bfloat16x2 store per plane.
__device__ __forceinline__ void split3_store2(__nv_bfloat16* o, int64_t plane, float x0, float x1) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const float r0 = __fsub_rn(x0, hf.x), r1 = __fsub_rn(x1, hf.y);
  const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
  const float2 mf = __bfloat1622float2(m);
  const __nv_bfloat162 l = __floats2bfloat162_rn(__fsub_rn(r0, mf.x), __fsub_rn(r1, mf.y));
  *reinterpret_cast<__nv_bfloat162*>(o) = h;
  *reinterpret_cast<__nv_bfloat162*>(o + plane) = m;
  *reinterpret_cast<__nv_bfloat162*>(o + 2 * plane) = l;
}

// Matvec input written next to a new basis vector.
constexpr int kInNone = 0;     // the matvec reads the FP64 basis vector itself
constexpr int kInPieces = 1;   // bfloat16 pieces of fl32(v), K-major [3][rows][Kp], zero in k >= cols
constexpr int kInF64 = 2;      // v as FP64 (double-float basis, FP64 matvec)

// Where a pass writes the shadow of the vector it writes: the hi and lo planes
// (hi == nullptr: no shadow; lo == nullptr: the hi plane only, the FP32
// truncation the pass-3 correction reads).
struct ShadowOut {
  float* hi;
  float* lo;
};

// two consecutive shadow elements (i even: one 8-byte store per plane)
__device__ __forceinline__ void store_shadow2(ShadowOut vs, int64_t i, double y0, double y1) {
  const float2 a = shadow_of(y0), b = shadow_of(y1);
  *reinterpret_cast<float2*>(vs.hi + i) = make_float2(a.x, b.x);
  if (vs.lo) *reinterpret_cast<float2*>(vs.lo + i) = make_float2(a.y, b.y);
}

template <class A, int MODE>
__device__ __forceinline__ void emit(typename A::V y, int64_t i, int64_t r, int64_t k, typename A::V* vn,
                                     __nv_bfloat16* pieces, int64_t Kp, int64_t plane, double* x64,
                                     ShadowOut vs = {nullptr, nullptr}) {
  vn[i] = y;
  if (vs.hi) {
    const float2 sh = shadow_of(A::to_double(y));
    vs.hi[i] = sh.x;
    if (vs.lo) vs.lo[i] = sh.y;
  }
  if (MODE == kInPieces) split3_store(pieces + r * Kp + k, plane, A::f32(y));
  if (MODE == kInF64) x64[i] = A::to_double(y);
}

// v_{j+1} = w / beta_j (unless stopped or gated off); element (r, k) of [rows][cols].
// vs (FP64 vectors, may be null): the double-float shadow of v_{j+1}.
template <class A, int MODE>
__global__ void __launch_bounds__(NT) k_next(const typename A::V* __restrict__ w, typename A::V* __restrict__ vn,
                                             int64_t rows, int64_t cols, __nv_bfloat16* __restrict__ pieces,
                                             int64_t Kp, double* __restrict__ x64, const double* __restrict__ scal,
                                             int j, const double* __restrict__ gate, ShadowOut vs) {
  if (scal[OFF_CTRL] != 0.0 || gate[0] != 0.0) return;
  const typename A::Coef c = A::coef(1.0 / scal[OFF_BETA + j]);
  const int64_t plane = rows * Kp;
  const int64_t kend = MODE == kInPieces ? Kp : cols;
  if constexpr (std::is_same<typename A::V, double>::value && MODE != kInF64) {
    if ((cols & 1) == 0) {   // element pairs: 16-byte loads and stores, bfloat16x2 pieces
      for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
        for (int64_t k = 2 * (int64_t)threadIdx.x; k < kend; k += 2 * NT) {
          if (k < cols) {
            const int64_t i = r * cols + k;
            const double2 x = *reinterpret_cast<const double2*>(w + i);
            const double y0 = A::mul(x.x, c), y1 = A::mul(x.y, c);
            *reinterpret_cast<double2*>(vn + i) = make_double2(y0, y1);
            if (vs.hi) store_shadow2(vs, i, y0, y1);
            if (MODE == kInPieces) split3_store2(pieces + r * Kp + k, plane, A::f32(y0), A::f32(y1));
          } else {
            split3_store2(pieces + r * Kp + k, plane, 0.f, 0.f);
          }
        }
      return;
    }
  }
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t k = threadIdx.x; k < kend; k += NT) {
      if (k < cols) {
        const int64_t i = r * cols + k;
        emit<A, MODE>(A::mul(w[i], c), i, r, k, vn, pieces, Kp, plane, x64, vs);
      } else {
        split3_store(pieces + r * Kp + k, plane, 0.f);
      }
    }
}

// Pass 3 folded into the next vector (FP64 vectors): v_{j+1} = (w - V h') /
// beta_j with the rounding-level terms h'_g v_g summed in FP32 (header);
// runs where k_post_pass2 chose it.  With the basis shadow (Vh: vector 0's hi
// plane, vector g's at Vh + g vh_ld) the FP32 basis values are read from its hi
// planes, which hold exactly f32_trunc of the basis, at half the bytes.
template <int MODE>
__global__ void __launch_bounds__(NT) k_next_corr(const double* __restrict__ V, int64_t ldv, int nv,
                                                  const double* __restrict__ w, double* __restrict__ vn, int64_t rows,
                                                  int64_t cols, __nv_bfloat16* __restrict__ pieces, int64_t Kp,
                                                  const double* __restrict__ scal, int j, ShadowOut vs,
                                                  const float* __restrict__ Vh, int64_t vh_ld) {
  if (scal[OFF_CTRL] != 0.0 || scal[OFF_LO + LO_GFAST] != 0.0) return;
  __shared__ float cf[MAXM];
  const double sc = scal[OFF_LO + LO_SC3];
  for (int g = threadIdx.x; g < nv; g += NT) cf[g] = (float)(scal[OFF_H2 + g] * sc);
  __syncthreads();
  const double isc = scal[OFF_LO + LO_ISC3];
  const double binv = 1.0 / scal[OFF_BETA + j];
  const int64_t plane = rows * Kp;
  const int64_t kend = MODE == kInPieces ? Kp : cols;
  if ((cols & 1) == 0) {   // element pairs: 16-byte loads and stores, bfloat16x2 pieces
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
      for (int64_t k = 2 * (int64_t)threadIdx.x; k < kend; k += 2 * NT) {
        if (k < cols) {
          const int64_t i = r * cols + k;
          float s0 = 0.f, s1 = 0.f;
          if (Vh) {
#pragma unroll 8
            for (int g = 0; g < nv; ++g) {
              const float2 v = *reinterpret_cast<const float2*>(Vh + (int64_t)g * vh_ld + i);
              s0 = __fmaf_rn(cf[g], v.x, s0);
              s1 = __fmaf_rn(cf[g], v.y, s1);
            }
          } else {
#pragma unroll 8
            for (int g = 0; g < nv; ++g) {
              const double2 v = *reinterpret_cast<const double2*>(V + (int64_t)g * ldv + i);
              s0 = __fmaf_rn(cf[g], f32_trunc(v.x), s0);
              s1 = __fmaf_rn(cf[g], f32_trunc(v.y), s1);
            }
          }
          const double2 x = *reinterpret_cast<const double2*>(w + i);
          const double y0 = fma(-(double)s0, isc, x.x) * binv, y1 = fma(-(double)s1, isc, x.y) * binv;
          *reinterpret_cast<double2*>(vn + i) = make_double2(y0, y1);
          if (vs.hi) store_shadow2(vs, i, y0, y1);
          if (MODE == kInPieces)
            split3_store2(pieces + r * Kp + k, plane, __double2float_rn(y0), __double2float_rn(y1));
        } else {
          split3_store2(pieces + r * Kp + k, plane, 0.f, 0.f);
        }
      }
    return;
  }
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t k = threadIdx.x; k < kend; k += NT) {
      if (k < cols) {
        const int64_t i = r * cols + k;
        float sf = 0.f;
        if (Vh) {
#pragma unroll 8
          for (int g = 0; g < nv; ++g) sf = __fmaf_rn(cf[g], Vh[(int64_t)g * vh_ld + i], sf);
        } else {
#pragma unroll 8
          for (int g = 0; g < nv; ++g) sf = __fmaf_rn(cf[g], f32_trunc(V[(int64_t)g * ldv + i]), sf);
        }
        const double y = fma(-(double)sf, isc, w[i]) * binv;
        emit<ArithF64, MODE>(y, i, r, k, vn, pieces, Kp, plane, nullptr, vs);
      } else {
        split3_store(pieces + r * Kp + k, plane, 0.f);
      }
    }
}

// v_0 = psi / ||psi|| (FP64 sum of squares already in scal[OFF_CTRL + 3])
template <class A, int MODE>
__global__ void __launch_bounds__(NT) k_start(const double* __restrict__ psi, typename A::V* __restrict__ v0,
                                              int64_t rows, int64_t cols, __nv_bfloat16* __restrict__ pieces,
                                              int64_t Kp, double* __restrict__ x64, const double* __restrict__ scal,
                                              ShadowOut vs) {
  const double inv = 1.0 / sqrt(scal[OFF_CTRL + 3]);
  const int64_t plane = rows * Kp;
  const int64_t kend = MODE == kInPieces ? Kp : cols;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t k = threadIdx.x; k < kend; k += NT) {
      if (k < cols) {
        const int64_t i = r * cols + k;
        emit<A, MODE>(A::from_double(psi[i] * inv), i, r, k, v0, pieces, Kp, plane, x64, vs);
      } else {
        split3_store(pieces + r * Kp + k, plane, 0.f);
      }
    }
}

template <class A>
__global__ void __launch_bounds__(NT) k_from_f64(const double* __restrict__ x, typename A::V* __restrict__ y, int64_t n,
                                                 const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
    y[i] = A::from_double(x[i]);
}

// x = sum_{j<k} y_j v_j (Ritz vector), stored as FP64
template <class A>
__global__ void __launch_bounds__(NT) k_ritz(const typename A::V* __restrict__ V, int64_t ldv,
                                             const double* __restrict__ scal, double* __restrict__ x, int64_t n) {
  __shared__ typename A::Coef ys[MAXM];
  const int k = (int)scal[OFF_CTRL + 1];
  for (int j = threadIdx.x; j < k; j += NT) ys[j] = A::coef(scal[OFF_Y + j]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
    typename A::Acc a = A::zero();
    for (int j = 0; j < k; ++j) A::acc_c(a, ys[j], V[(int64_t)j * ldv + i]);
    x[i] = A::value(a);
  }
}

// ---------------------------------------------------------------- scalar kernels
// out[v] = sum_{b < nb} part[v*NBMAX + b] in order; one block per vector.
__global__ void k_reduce_parts(const double* __restrict__ part, int nv, int nb, double* __restrict__ out,
                               const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  const int v = blockIdx.x;
  if (v >= nv) return;
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(int64_t)v * NBMAX + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    out[v] = r;
  }
}

// FP64 partial sums of squares of psi (the start vector's norm)
__global__ void __launch_bounds__(NT) k_sumsq(const double* __restrict__ w, int64_t n, double* __restrict__ part) {
  __shared__ double sh[NT / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) acc = fma(w[i], w[i], acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < NT / 32; ++k) s += sh[k];
    part[blockIdx.x] = s;
  }
}

// alpha_j = <v_j, H v_j> (the pass-1 coefficient of v_j); without
// re-orthogonalisation the pass-3 coefficients are (beta_{j-1}, alpha_j).
// With dgks, the second Gram-Schmidt pass is kept only where the first one
// cancelled: ||w'||^2 = ||w||^2 - sum_i h_i^2 (V orthonormal) below
// ||w||^2 / 2, i.e. ||w'|| < ||w|| / sqrt(2) (Daniel, Gragg, Kaufman & Stewart,
// Math. Comp. 30, 1976).  Gates read by the passes that follow (a pass runs
// while its gate is 0): ctrl[5] = 1 when the second pass is skipped (or the
// iteration stopped), ctrl[6] = 1 when it is taken (or stopped).
//
// With f32 (FP64 vectors, re-orthogonalisation) the terms of h_0 .. h_{j-2}
// in passes 2 and 2' are summed in FP32 where sum |h_i| (j + 7) <= 2^-32 ||w||,
// else in double-float where it is <= 2^-10 ||w|| and j >= 7 (header); the
// scale puts the largest of them in [1, 2).
__global__ void k_post_pass1(double* scal, int j, int reorth, int dgks, int f32) {
  double* ctrl = scal + OFF_CTRL;
  double* lo = scal + OFF_LO;
  lo[LO_NS1] = 0.0;
  if (ctrl[0] != 0.0) {
    ctrl[5] = 1.0;
    ctrl[6] = 1.0;
    return;
  }
  scal[OFF_ALPHA + j] = scal[OFF_H + j];
  if (!reorth && j > 0) scal[OFF_H + j - 1] = scal[OFF_BETA + j - 1];
  bool second = true;
  if (reorth && dgks) {
    double h2 = 0.0;
    for (int i = 0; i <= j; ++i) h2 += scal[OFF_H + i] * scal[OFF_H + i];
    second = ctrl[4] - h2 < 0.5 * ctrl[4];
  }
  ctrl[5] = second ? 0.0 : 1.0;
  ctrl[6] = second ? 1.0 : 0.0;
  if (reorth && second) ctrl[7] += 1.0;   // second passes taken (reported with TCI_VERBOSE)
  if (reorth && f32 && j >= 2) {
    double l1 = 0.0, mx = 0.0;
    for (int i = 0; i + 1 < j; ++i) {
      const double a = fabs(scal[OFF_H + i]);
      l1 += a;
      mx = fmax(mx, a);
    }
    const double wn = sqrt(ctrl[4]), k8 = (double)(j + 7);
    // double-float terms only from six terms on (fewer cost more than their FP64 FMAs)
    const int mode = l1 * k8 <= kF32Bound * wn ? kTermsF32 : (j >= 7 && l1 * k8 <= kDFBound * wn) ? kTermsDF : kTermsF64;
    if (mode != kTermsF64) {
      const int e = mx > 0.0 ? ilogb(mx) : 0;
      lo[LO_NS1] = (double)(j - 1);
      lo[LO_MODE1] = (double)mode;
      lo[LO_SC1] = ldexp(1.0, -e);
      lo[LO_ISC1] = ldexp(1.0, e);
      lo[mode == kTermsF32 ? LO_N1 : LO_N2] += 1.0;
    }
  }
}

// After pass 2 (second Gram-Schmidt pass taken and not stopped): fold pass 3
// into the next-vector kernel where f32 and sum |h'_i| (j + 9) <= 2^-32 ||w'||,
// setting ||w||^2 = ||w'||^2 - |h'|^2 for beta_j; else run pass 3 in FP64.
// Gates (run while 0): LO_GFAST fused kernel, LO_GSLOW FP64 pass 3,
// LO_GNEXT plain next-vector kernel.
__global__ void k_post_pass2(double* scal, int j, int f32) {
  double* ctrl = scal + OFF_CTRL;
  double* lo = scal + OFF_LO;
  if (ctrl[0] != 0.0 || ctrl[5] != 0.0) {   // stopped, or the second pass was skipped
    lo[LO_GFAST] = 1.0;
    lo[LO_GSLOW] = 1.0;
    lo[LO_GNEXT] = 0.0;
    return;
  }
  double l1 = 0.0, l2 = 0.0, mx = 0.0;
  for (int i = 0; i <= j; ++i) {
    const double a = fabs(scal[OFF_H2 + i]);
    l1 += a;
    l2 += a * a;
    mx = fmax(mx, a);
  }
  const double wn2 = lo[LO_WN2];
  const bool fast = f32 && wn2 > 0.0 && l1 * (double)(j + 9) <= kF32Bound * sqrt(wn2);
  lo[LO_GFAST] = fast ? 0.0 : 1.0;
  lo[LO_GSLOW] = fast ? 1.0 : 0.0;
  lo[LO_GNEXT] = fast ? 1.0 : 0.0;
  if (fast) {
    const int e = mx > 0.0 ? ilogb(mx) : 0;
    lo[LO_SC3] = ldexp(1.0, -e);
    lo[LO_ISC3] = ldexp(1.0, e);
    ctrl[3] = wn2 - l2;
    lo[LO_N3] += 1.0;
  }
}

// beta_j = ||w||, stop test, step counter.
__global__ void k_finish_beta(double* scal, int j, int m, double tol) {
  if (scal[OFF_CTRL] != 0.0) return;
  const double b = sqrt(scal[OFF_CTRL + 3]);
  const double a = scal[OFF_ALPHA + j];
  scal[OFF_BETA + j] = b;
  scal[OFF_CTRL + 1] = (double)(j + 1);
  if (j == m - 1 || b < tol * fabs(a)) scal[OFF_CTRL] = 1.0;
}

// Negative LDL^T pivots of T - x I = eigenvalues of T below x (Sylvester
// inertia); a zero pivot is replaced by a tiny negative value as soon as it
// appears, so it is counted and divides the next pivot.
__device__ int sturm_count(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < m; ++i) {
    q = i == 0 ? a[0] - x : a[i] - x - b[i - 1] * b[i - 1] / q;
    if (q == 0.0) q = -2.2250738585072014e-308;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// K7: lowest eigenpair of T_k = tridiag(beta, alpha, beta) in one warp:
// multisection on the Sturm count (each of kTriP threads tests one point per
// round), then inverse iteration with Gaussian elimination with partial
// pivoting on T - sigma I.  One warp, not a block: every Sturm count costs m
// FP64 divisions, which B300's FP64 pipe makes the expensive part (256 points
// per round took ~76 us per solve; 32 points need ~2x the rounds at 1/8 the
// divisions each).
constexpr int kTriP = 32;
__global__ void __launch_bounds__(kTriP) k_tridiag_lowest(double* scal) {
  __shared__ double a[MAXM], b[MAXM];
  __shared__ double lo, hi;
  __shared__ int first;
  const int m = (int)scal[OFF_CTRL + 1];
  if (m <= 0) return;
  for (int i = threadIdx.x; i < m; i += kTriP) {
    a[i] = scal[OFF_ALPHA + i];
    b[i] = i < m - 1 ? scal[OFF_BETA + i] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double l = 1e300, h = -1e300;
    for (int i = 0; i < m; ++i) {
      double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
      l = fmin(l, a[i] - r);
      h = fmax(h, a[i] + r);
    }
    lo = l;
    hi = h;
  }
  __syncthreads();
  for (int round = 0; round < 256; ++round) {   // ends at an ulp long before (33x per round)
    const double l = lo, h = hi;
    const double x = l + (h - l) * (double)(threadIdx.x + 1) / (double)(kTriP + 1);
    if (threadIdx.x == 0) first = kTriP;
    __syncthreads();
    const bool hit = x > l && x < h && sturm_count(a, b, m, x) >= 1;
    if (hit) atomicMin(&first, (int)threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int f = first;
      double nl = l, nh = h;
      if (f < kTriP) {
        nh = l + (h - l) * (double)(f + 1) / (double)(kTriP + 1);
        if (f > 0) nl = l + (h - l) * (double)f / (double)(kTriP + 1);
      } else {
        nl = l + (h - l) * (double)kTriP / (double)(kTriP + 1);
      }
      if (!(nl > l) && !(nh < h)) {   // no progress: converged to an ulp
        nl = l;
        nh = h;
        first = -1;
      }
      lo = nl;
      hi = nh;
    }
    __syncthreads();
    if (first == -1) break;
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double theta = 0.5 * (lo + hi);
  scal[OFF_CTRL + 2] = theta;
  // inverse iteration
  const double sigma = theta - 1e-10 * fmax(1.0, fabs(theta));
  double d[MAXM], du[MAXM], du2[MAXM], dl[MAXM], y[MAXM];
  int piv[MAXM];
  for (int i = 0; i < m; ++i) {
    d[i] = a[i] - sigma;
    du[i] = b[i];
    dl[i] = b[i];
    du2[i] = 0.0;
    y[i] = 1.0 / sqrt((double)m);
  }
  for (int i = 0; i < m - 1; ++i) {
    if (fabs(d[i]) >= fabs(dl[i])) {
      if (d[i] == 0.0) d[i] = 1e-300;
      const double f = dl[i] / d[i];
      dl[i] = f;
      d[i + 1] -= f * du[i];
      piv[i] = 0;
    } else {
      const double f = d[i] / dl[i];
      d[i] = dl[i];
      dl[i] = f;
      const double t = du[i];
      du[i] = d[i + 1];
      d[i + 1] = t - f * d[i + 1];
      if (i < m - 2) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du[i + 1];
      }
      piv[i] = 1;
    }
  }
  if (d[m - 1] == 0.0) d[m - 1] = 1e-300;
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i < m - 1; ++i) {
      if (piv[i]) {
        const double t = y[i];
        y[i] = y[i + 1];
        y[i + 1] = t - dl[i] * y[i];
      } else {
        y[i + 1] -= dl[i] * y[i];
      }
    }
    y[m - 1] /= d[m - 1];
    if (m > 1) y[m - 2] = (y[m - 2] - du[m - 2] * y[m - 1]) / d[m - 2];
    for (int i = m - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / d[i];
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += y[i] * y[i];
    nrm = 1.0 / sqrt(nrm);
    for (int i = 0; i < m; ++i) y[i] *= nrm;
  }
  int kmax = 0;
  for (int i = 1; i < m; ++i)
    if (fabs(y[i]) > fabs(y[kmax])) kmax = i;
  const double sgn = y[kmax] > 0 ? 1.0 : -1.0;
  for (int i = 0; i < m; ++i) scal[OFF_Y + i] = sgn * y[i];
}

// ---------------------------------------------------------------- short vectors
// One step's vector work for short FP64 vectors (re-orthogonalisation, the
// matvec reading the basis itself) in a single launch of one cluster of
// up to kSmallClMax CTAs: pass 1 (dots, ||w||^2), the DGKS test, pass 2 (update, and
// where the second pass is taken its dots), pass 3, beta_j, the stop test
// and v_{j+1}, each pass's block sums combined across the cluster through
// distributed shared memory.  Every thread owns the same elements in every
// pass, and every CTA adds the CTAs' sums in rank order, so the totals are
// identical in all CTAs and deterministic.  Used where n (j + 2) is small
// enough that launches, not FP64 FMAs, set the step's time; it writes the
// same scalars and vectors as the multi-kernel path, so the two mix freely
// from step to step.
namespace cg = cooperative_groups;
constexpr int kSmallClMax = 16, kSmallNT = 512;
constexpr int64_t kSmallWork = 1 << 19;   // n (j + 2) up to which a step runs as one launch

__global__ void __launch_bounds__(kSmallNT)
    k_step_small(double* __restrict__ V, int64_t ldv, double* __restrict__ w, int64_t n,
                 double* __restrict__ scal, int j, int m, double tol, int dgks) {
  double* ctrl = scal + OFF_CTRL;
  if (ctrl[0] != 0.0) return;   // stopped: every CTA reads the same flag and leaves together
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double part[MAXM + 2], tot[MAXM + 2], hs[MAXM + 1];
  __shared__ double wred[kSmallNT / 32][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ncl = (int)cl.num_blocks();
  const int64_t T = (int64_t)ncl * kSmallNT;
  const int64_t t0 = (int64_t)cl.block_rank() * kSmallNT + threadIdx.x;
  const int nv = j + 1;

  // block sums of a[0..cnt) into part[base..base+cnt)
  auto block_sum8 = [&](const double (&a)[8], int base, int cnt) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double v = warp_sum(a[k]);
      if (lane == 0) wred[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double v = 0.0;
      for (int q = 0; q < kSmallNT / 32; ++q) v += wred[q][threadIdx.x];
      part[base + threadIdx.x] = v;
    }
    __syncthreads();
  };
  // cluster totals of part[0..cnt) into tot, in rank order
  auto cluster_sum = [&](int cnt) {
    cl.sync();
    for (int k = threadIdx.x; k < cnt; k += kSmallNT) {
      double v = 0.0;
      for (int r = 0; r < ncl; ++r) v += cl.map_shared_rank(part, r)[k];
      tot[k] = v;
    }
    cl.sync();   // all remote reads done before part is rewritten; tot visible block-wide
  };
  // sums over the owned elements of: dots <V_g, w> for g < ndot, then (sq) ||w||^2
  auto dots = [&](int ndot, bool sq) {
    const int nval = ndot + (sq ? 1 : 0);
    for (int g0 = 0; g0 < nval; g0 += 8) {
      double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int64_t i = t0; i < n; i += T) {
        const double x = w[i];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int g = g0 + k;
          if (g < ndot) a[k] = fma(V[(int64_t)g * ldv + i], x, a[k]);
          else if (g == ndot && sq) a[k] = fma(x, x, a[k]);
        }
      }
      block_sum8(a, g0, nval - g0 < 8 ? nval - g0 : 8);
    }
    cluster_sum(nval);
  };
  // w -= sum_g c_g V_g over the owned elements, then the cluster total of ||w||^2 in tot[0]
  auto update_sq = [&](const double* c) {
    double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = t0; i < n; i += T) {
      double sacc = 0.0;
      for (int g = 0; g < nv; ++g) sacc = fma(c[g], V[(int64_t)g * ldv + i], sacc);
      const double y = w[i] - sacc;
      w[i] = y;
      a[0] = fma(y, y, a[0]);
    }
    block_sum8(a, 0, 1);
    cluster_sum(1);
  };

  dots(nv, true);                                    // pass 1: h = V^T w, ||w||^2
  for (int g = threadIdx.x; g < nv; g += kSmallNT) hs[g] = tot[g];
  const double wn2_1 = tot[nv];
  __syncthreads();
  const double alpha = hs[j];
  double hh = 0.0;
  for (int g = 0; g < nv; ++g) hh += hs[g] * hs[g];
  const bool second = !dgks || wn2_1 - hh < 0.5 * wn2_1;   // DGKS test, as k_post_pass1
  double wn2;
  if (second) {
    update_sq(hs);                                   // pass 2: w -= V h (its norm unused)
    dots(nv, false);                                 // h' = V^T w
    __syncthreads();
    for (int g = threadIdx.x; g < nv; g += kSmallNT) hs[g] = tot[g];
    __syncthreads();
    update_sq(hs);                                   // pass 3: w -= V h', ||w||^2
  } else {
    update_sq(hs);                                   // pass 2': w -= V h, ||w||^2
  }
  wn2 = tot[0];
  const double b = sqrt(wn2);
  const bool stop = j == m - 1 || b < tol * fabs(alpha);   // as k_finish_beta
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    scal[OFF_H + j] = alpha;
    scal[OFF_ALPHA + j] = alpha;
    scal[OFF_BETA + j] = b;
    ctrl[1] = (double)(j + 1);
    ctrl[3] = wn2;
    ctrl[4] = wn2_1;
    if (second) ctrl[7] += 1.0;
    if (stop) ctrl[0] = 1.0;
  }
  if (!stop) {                                       // v_{j+1} = w / beta_j
    const double inv = 1.0 / b;
    double* vn = V + (int64_t)(j + 1) * ldv;
    for (int64_t i = t0; i < n; i += T) vn[i] = w[i] * inv;
  }
}

__global__ void k_init_scal(double* scal) {
  for (int i = threadIdx.x; i < NSCAL; i += blockDim.x) scal[i] = 0.0;
}


}  // namespace

// ---------------------------------------------------------------- host side
namespace {

// Grid of a vector pass: one full wave, i.e. the SM count times the blocks
// of NT threads that fit on one SM (from the kernel's registers and shared
// memory), capped at NBMAX partial-sum slots.  Fixed per kernel and device,
// so the reductions stay deterministic.
int wave_grid(tci_context ctx, const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, ctx->device);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, NT, 0) != cudaSuccess || occ < 1) occ = 1;
  int g = occ * ctx->num_sms;
  if (g > NBMAX) g = NBMAX;
  cache[key] = g;
  return g;
}

// Grid of a vector pass over n elements: one wave, but no more blocks than
// give each thread 8 elements (short vectors, e.g. DMRG bonds of small chi,
// would otherwise spend the pass on empty blocks and a long partial-sum
// reduction).  Fixed per (kernel, device, n), so reductions stay deterministic.
int pass_grid(tci_context ctx, const void* kernel, int64_t n) {
  const int g = wave_grid(ctx, kernel);
  const int64_t cap = (n + (int64_t)NT * 8 - 1) / ((int64_t)NT * 8);
  return cap < g ? (int)(cap < 1 ? 1 : cap) : g;
}

template <class A, int G, bool SQ>
int dots_launch_g(tci_context ctx, const typename A::V* V, int64_t ldv, int v0, int nv, const typename A::V* w,
                  int64_t n, double* part, double* part_sq, const double* ctrl, const PassOut& po) {
  const int grid = pass_grid(ctx, (const void*)k_dots<A, G, SQ>, n);
  k_dots<A, G, SQ><<<grid, NT, 0, ctx->stream>>>(V, ldv, v0, nv, w, n, part, part_sq, ctrl, po);
  return grid;
}

// FP64 passes are instantiated for every basis size G = nv: the compiler
// evaluates the FMAs of an unrolled `if (g < nv)` loop unconditionally and
// selects the result, and on B300 each needless DFMA costs as much as a
// needed one.  Double-float passes (FP32 pipes) use G in {8, 16, GMAX}.
template <class A, bool SQ, int G = 1>
int dots_exact(tci_context ctx, const typename A::V* V, int64_t ldv, int v0, int nv, const typename A::V* w,
               int64_t n, double* part, double* part_sq, const double* ctrl, const PassOut& po) {
  if constexpr (G == GMAX) {
    return dots_launch_g<A, GMAX, SQ>(ctx, V, ldv, v0, nv, w, n, part, part_sq, ctrl, po);
  } else {
    if (nv <= G) return dots_launch_g<A, G, SQ>(ctx, V, ldv, v0, nv, w, n, part, part_sq, ctrl, po);
    return dots_exact<A, SQ, G + 1>(ctx, V, ldv, v0, nv, w, n, part, part_sq, ctrl, po);
  }
}

template <class A, bool SQ>
int dots_launch(tci_context ctx, const typename A::V* V, int64_t ldv, int v0, int nv, const typename A::V* w,
                int64_t n, double* part, double* part_sq, const double* ctrl, const PassOut& po) {
  if constexpr (std::is_same<A, ArithF64>::value) {
    return dots_exact<A, SQ>(ctx, V, ldv, v0, nv, w, n, part, part_sq, ctrl, po);
  } else {
    if (nv <= 8) return dots_launch_g<A, 8, SQ>(ctx, V, ldv, v0, nv, w, n, part, part_sq, ctrl, po);
    if (nv <= 16) return dots_launch_g<A, 16, SQ>(ctx, V, ldv, v0, nv, w, n, part, part_sq, ctrl, po);
    return dots_launch_g<A, GMAX, SQ>(ctx, V, ldv, v0, nv, w, n, part, part_sq, ctrl, po);
  }
}

// out[0..nv) = <V_{v0+v}, w>; *sumsq_out = ||w||^2 when sumsq_out.  With a
// ticket (a zero unsigned in device memory) each pass's last block forms the
// totals; without, k_reduce_parts launches do.
template <class A>
tci_status run_dots(tci_context ctx, const typename A::V* V, int64_t ldv, int v0, int nv, const typename A::V* w,
                    int64_t n, double* part, double* out, const double* ctrl, double* sumsq_out = nullptr,
                    unsigned* ticket = nullptr) {
  double* part_sq = part + (int64_t)MAXM * NBMAX;
  for (int g0 = 0; g0 < nv; g0 += GMAX) {
    const int g = nv - g0 < GMAX ? nv - g0 : GMAX;
    const bool sq = sumsq_out && g0 == 0;
    PassOut po;
    if (ticket) po = {out + g0, sq ? sumsq_out : nullptr, ticket};
    const int grid = sq ? dots_launch<A, true>(ctx, V, ldv, v0 + g0, g, w, n, part, part_sq, ctrl, po)
                        : dots_launch<A, false>(ctx, V, ldv, v0 + g0, g, w, n, part, part_sq, ctrl, po);
    if (ticket) continue;
    k_reduce_parts<<<g, 256, 0, ctx->stream>>>(part + (int64_t)(v0 + g0) * NBMAX, g, grid, out + g0, ctrl);
    if (sq) k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part_sq, 1, grid, sumsq_out, ctrl);
  }
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

template <int G, bool SQ>
int dots_shadow_g(tci_context ctx, const float* Vs, int64_t ldv, int nv, const double* w, int64_t n, double* part,
                  double* part_sq, const double* ctrl) {
  const int grid = pass_grid(ctx, (const void*)k_dots_shadow<G, SQ>, n);
  k_dots_shadow<G, SQ><<<grid, NT, 0, ctx->stream>>>(Vs, ldv, nv, w, n, part, part_sq, ctrl);
  return grid;
}

template <bool SQ>
int dots_shadow_launch(tci_context ctx, const float* Vs, int64_t ldv, int nv, const double* w, int64_t n,
                       double* part, double* part_sq, const double* ctrl) {
  if (nv <= 4) return dots_shadow_g<4, SQ>(ctx, Vs, ldv, nv, w, n, part, part_sq, ctrl);
  if (nv <= 8) return dots_shadow_g<8, SQ>(ctx, Vs, ldv, nv, w, n, part, part_sq, ctrl);
  if (nv <= 12) return dots_shadow_g<12, SQ>(ctx, Vs, ldv, nv, w, n, part, part_sq, ctrl);
  if (nv <= 16) return dots_shadow_g<16, SQ>(ctx, Vs, ldv, nv, w, n, part, part_sq, ctrl);
  return dots_shadow_g<GMAX, SQ>(ctx, Vs, ldv, nv, w, n, part, part_sq, ctrl);
}

// run_dots (v0 = 0) from the basis shadow
tci_status run_dots_shadow(tci_context ctx, const float* Vs, int64_t ldv, int nv, const double* w, int64_t n,
                           double* part, double* out, const double* ctrl, double* sumsq_out) {
  double* part_sq = part + (int64_t)MAXM * NBMAX;
  for (int g0 = 0; g0 < nv; g0 += GMAX) {
    const int g = nv - g0 < GMAX ? nv - g0 : GMAX;
    const bool sq = sumsq_out && g0 == 0;
    const float* Vb = Vs + 2 * (int64_t)g0 * ldv;
    double* pb = part + (int64_t)g0 * NBMAX;
    const int grid = sq ? dots_shadow_launch<true>(ctx, Vb, ldv, g, w, n, pb, part_sq, ctrl)
                        : dots_shadow_launch<false>(ctx, Vb, ldv, g, w, n, pb, part_sq, ctrl);
    k_reduce_parts<<<g, 256, 0, ctx->stream>>>(pb, g, grid, out + g0, ctrl);
    if (sq) k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part_sq, 1, grid, sumsq_out, ctrl);
  }
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

// Every variant of one pass uses the grid of its FP64 variant, so the partial
// sums of whichever variant ran are reduced over the same block count.
template <class A, int G, bool DOTS, bool SUMSQ, int TERMS>
int update_launch_g(tci_context ctx, const typename A::V* V, int64_t ldv, int v0, int nv, const double* coef,
                    typename A::V* w, int64_t n, double* part, double* part_sq, const double* ctrl,
                    const double* lo, const PassOut& po) {
  const int grid = pass_grid(ctx, (const void*)k_update<A, G, DOTS, SUMSQ, kTermsF64>, n);
  k_update<A, G, DOTS, SUMSQ, TERMS><<<grid, NT, 0, ctx->stream>>>(V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl,
                                                                  lo, po);
  return grid;
}

template <int G, bool DOTS, bool SUMSQ, bool DFD>
int update_sel_g(tci_context ctx, const double* V, int64_t ldv, int v0, int nv, const double* coef, double* w,
                 int64_t n, double* part, double* part_sq, const double* ctrl, const double* lo, const PassOut& po) {
  const int grid = pass_grid(ctx, (const void*)k_update_sel<G, DOTS, SUMSQ, DFD>, n);
  k_update_sel<G, DOTS, SUMSQ, DFD><<<grid, NT, 0, ctx->stream>>>(V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
  return grid;
}

template <bool DOTS, bool SUMSQ, bool DFD, int G = 3>
int update_sel(tci_context ctx, const double* V, int64_t ldv, int v0, int nv, const double* coef, double* w,
               int64_t n, double* part, double* part_sq, const double* ctrl, const double* lo, const PassOut& po) {
  if constexpr (G == GMAX) {
    return update_sel_g<GMAX, DOTS, SUMSQ, DFD>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
  } else {
    if (nv <= G) return update_sel_g<G, DOTS, SUMSQ, DFD>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
    return update_sel<DOTS, SUMSQ, DFD, G + 1>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
  }
}

template <class A, bool DOTS, bool SUMSQ, int TERMS, int G = 1>
int update_exact(tci_context ctx, const typename A::V* V, int64_t ldv, int v0, int nv, const double* coef,
                 typename A::V* w, int64_t n, double* part, double* part_sq, const double* ctrl, const double* lo, const PassOut& po) {
  if constexpr (G == GMAX) {
    return update_launch_g<A, GMAX, DOTS, SUMSQ, TERMS>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
  } else {
    if (nv <= G)
      return update_launch_g<A, G, DOTS, SUMSQ, TERMS>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
    return update_exact<A, DOTS, SUMSQ, TERMS, G + 1>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
  }
}

// One update pass; with lo (FP64 vectors, more than two terms) one launch
// runs the term arithmetic the device chose (k_update_sel).  df_dots: the
// double-float-terms variant forms its dots in double-float.
template <class A, bool DOTS, bool SUMSQ>
int update_launch(tci_context ctx, const typename A::V* V, int64_t ldv, int v0, int nv, const double* coef,
                  typename A::V* w, int64_t n, double* part, double* part_sq, const double* ctrl, const double* lo,
                  bool df_dots, const PassOut& po) {
  if constexpr (std::is_same<A, ArithF64>::value) {
    if (lo && nv > 2) {
      if (DOTS && df_dots) return update_sel<DOTS, SUMSQ, true>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
      return update_sel<DOTS, SUMSQ, false>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
    }
    return update_exact<A, DOTS, SUMSQ, kTermsF64>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
  } else {
    if (nv <= 8)
      return update_launch_g<A, 8, DOTS, SUMSQ, kTermsF64>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
    if (nv <= 16)
      return update_launch_g<A, 16, DOTS, SUMSQ, kTermsF64>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
    return update_launch_g<A, GMAX, DOTS, SUMSQ, kTermsF64>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, po);
  }
}

// w -= sum_{v0 <= v < v0+nv} coef[v] V_v; then dots_out[0..nv) = <V_v, w>
// (when dots_out) and *sumsq_out = ||w||^2 (when sumsq_out).  One fused pass
// for nv <= GMAX (with lo: FP32 rounding-level terms, v0 = 0); a larger
// basis is updated group by group in FP64 and its dots taken in a separate pass.
template <class A>
tci_status run_update(tci_context ctx, const typename A::V* V, int64_t ldv, int v0, int nv, const double* coef,
                      typename A::V* w, int64_t n, double* part, double* dots_out, double* sumsq_out,
                      const double* ctrl, const double* lo = nullptr, bool df_dots = false,
                      unsigned* ticket = nullptr) {
  double* part_sq = part + (int64_t)MAXM * NBMAX;
  if (lo && v0 != 0) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "lanczos: internal (FP32 terms need v0 = 0)");
  int sq_grid = 0;
  if (nv <= GMAX) {
    PassOut po;
    if (ticket && (dots_out || sumsq_out)) po = {dots_out, sumsq_out, ticket};
    int grid = 0;
    if (dots_out && sumsq_out)
      grid = update_launch<A, true, true>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, df_dots, po);
    else if (dots_out)
      grid = update_launch<A, true, false>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, df_dots, po);
    else if (sumsq_out)
      grid = update_launch<A, false, true>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, false, po);
    else
      update_launch<A, false, false>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl, lo, false, po);
    if (ticket) sumsq_out = nullptr;   // reduced by the pass's last block
    else if (dots_out)
      k_reduce_parts<<<nv, 256, 0, ctx->stream>>>(part + (int64_t)v0 * NBMAX, nv, grid, dots_out, ctrl);
    sq_grid = grid;
  } else {
    for (int g0 = 0; g0 < nv; g0 += GMAX) {
      const int g = nv - g0 < GMAX ? nv - g0 : GMAX;
      if (g0 + g == nv && sumsq_out && !dots_out) {
        PassOut po;
        if (ticket) po = {nullptr, sumsq_out, ticket};
        sq_grid = update_launch<A, false, true>(ctx, V, ldv, v0 + g0, g, coef, w, n, part, part_sq, ctrl, nullptr,
                                                false, po);
        if (ticket) sumsq_out = nullptr;
      } else {
        update_launch<A, false, false>(ctx, V, ldv, v0 + g0, g, coef, w, n, part, part_sq, ctrl, nullptr, false,
                                       PassOut{});
      }
    }
    if (dots_out) {
      TCI_TRY(run_dots<A>(ctx, V, ldv, v0, nv, w, n, part, dots_out, ctrl, sumsq_out, ticket));
      sumsq_out = nullptr;   // reduced by run_dots
    }
  }
  if (sumsq_out) k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part_sq, 1, sq_grid, sumsq_out, ctrl);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

template <class A, int MODE>
void launch_start(tci_context ctx, const double* psi0, typename A::V* v0, int64_t rows, int64_t cols,
                  __nv_bfloat16* pieces, int64_t Kp, double* x64, const double* S, ShadowOut vs) {
  const int blocks = (int)(rows < (int64_t)NBMAX * 8 ? rows : (int64_t)NBMAX * 8);
  k_start<A, MODE><<<blocks, NT, 0, ctx->stream>>>(psi0, v0, rows, cols, pieces, Kp, x64, S, vs);
}

template <class A, int MODE>
void launch_next(tci_context ctx, const typename A::V* w, typename A::V* vn, int64_t rows, int64_t cols,
                 __nv_bfloat16* pieces, int64_t Kp, double* x64, const double* S, int j, const double* gate,
                 ShadowOut vs) {
  const int blocks = (int)(rows < (int64_t)NBMAX * 8 ? rows : (int64_t)NBMAX * 8);
  k_next<A, MODE><<<blocks, NT, 0, ctx->stream>>>(w, vn, rows, cols, pieces, Kp, x64, S, j, gate, vs);
}

template <int MODE>
void launch_next_corr(tci_context ctx, const double* V, int64_t ldv, int nv, const double* w, double* vn,
                      int64_t rows, int64_t cols, __nv_bfloat16* pieces, int64_t Kp, const double* S, int j,
                      ShadowOut vs, const float* Vh, int64_t vh_ld) {
  const int blocks = (int)(rows < (int64_t)NBMAX * 8 ? rows : (int64_t)NBMAX * 8);
  k_next_corr<MODE><<<blocks, NT, 0, ctx->stream>>>(V, ldv, nv, w, vn, rows, cols, pieces, Kp, S, j, vs, Vh, vh_ld);
}

// One cluster of the largest size the device runs (16 CTAs where
// non-portable cluster sizes are allowed, else 8), found once per device.
int small_cluster(tci_context ctx) {
  static std::mutex mu;
  static std::map<int, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(ctx->device);
  if (it != cache.end()) return it->second;
  int best = 8;
  if (cudaFuncSetAttribute(k_step_small, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kSmallClMax;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kSmallClMax);
    cfg.blockDim = dim3(kSmallNT);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_step_small, &cfg) == cudaSuccess && nclusters >= 1)
      best = kSmallClMax;
  }
  cudaGetLastError();
  cache[ctx->device] = best;
  return best;
}

tci_status launch_step_small(tci_context ctx, double* V, int64_t ldv, double* w, int64_t n, double* S, int j,
                             int nsteps, double tol, int dgks) {
  const int ncl = small_cluster(ctx);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ncl);
  cfg.blockDim = dim3(kSmallNT);
  cfg.stream = ctx->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  TCI_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_step_small, V, ldv, w, n, S, j, nsteps, tol, dgks));
  return TCI_OK;
}

// The Lanczos iteration in arithmetic A with matvec input mode MODE
// (kInPieces for a split-BF16 plan; kInNone for FP64 vectors on an FP64
// plan; kInF64 for double-float vectors on an FP64 plan).
template <class A, int MODE>
// Vs (FP64 vectors on a split plan, re-orthogonalised; else null): a copy of
// the basis written with each basis vector.  The pass-3 correction reads its
// hi planes (the FP32 truncation its rounding-level terms use: half the bytes
// of the FP64 basis; vector g's at Vs + g ldv).  With dfdots each vector also
// has a lo plane (vector g: hi at Vs + 2 g ldv, lo ldv after it) and pass 1
// and the second pass's dots run in double-float from the copy.
tci_status lanczos_run(tci_heff_plan p, const double* psi0, int nsteps, int reorth, double* x, double tol,
                       float* Vs, bool dfdots) {
  using Vt = typename A::V;
  tci_context ctx = p->ctx;
  // a complex plan runs on the real form: C128 vectors as interleaved FP64 pairs
  const int64_t rows = p->cplx ? 2 * p->chiL * p->cd * p->cd : p->chiL * 4, cols = p->chiR;
  const int64_t n = rows * cols;
  const int64_t ldv = (n + 31) / 32 * 32;
  constexpr bool kDF = std::is_same<Vt, float2>::value;
  // FP32 rounding-level terms: FP64 vectors whose next vector is written by
  // k_next / k_next_corr (every mode but the double-float one)
  constexpr bool kF32Terms = !kDF && MODE != kInF64;
  if (MODE == kInF64) {
    if (!p->lz_x64) TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * n, (void**)&p->lz_x64));
    if (!p->lz_o64) TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * n, (void**)&p->lz_o64));
  }
  double* S = p->lz_scal;
  double* ctrl = S + OFF_CTRL;
  Vt* V = (Vt*)p->lz_V;
  Vt* w = (Vt*)p->lz_w;
  double* part = p->lz_part;
  __nv_bfloat16* pieces = MODE == kInPieces ? (__nv_bfloat16*)p->psip : nullptr;
  const int64_t Kp = MODE == kInPieces ? p->Kp1 : 0;

  k_init_scal<<<1, 256, 0, ctx->stream>>>(S);
  // blocks-done counter of the passes whose last block forms the totals (zeroed with S)
  unsigned* ticket = reinterpret_cast<unsigned*>(S + OFF_TICKET);
  k_sumsq<<<NBMAX, NT, 0, ctx->stream>>>(psi0, n, part);
  k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part, 1, NBMAX, ctrl + 3, ctrl);
  if (kDF || !reorth) Vs = nullptr;
  if (!Vs) dfdots = false;
  const int64_t vs_ld = dfdots ? 2 * ldv : ldv;   // between consecutive vectors' hi planes
  launch_start<A, MODE>(ctx, psi0, V, rows, cols, pieces, Kp, p->lz_x64, S,
                        ShadowOut{Vs, dfdots ? Vs + ldv : nullptr});
  TCI_CUDA(ctx, cudaGetLastError());
  for (int j = 0; j < nsteps; ++j) {
    Vt* vj = V + (int64_t)j * ldv;
    // split plan, FP64 vectors: the first projection's dots h = V^T w and ||w||^2
    // come out of the matvec's GEMM2 epilogue (per-CTA partials, reduced in order)
    const bool fused = MODE == kInPieces && !kDF && reorth && p->lz_fuse && j + 1 <= kFusedMax;
    // w = H v_j
    if (fused) {
      int grid = 0;
      TCI_TRY(tci_heff_apply_raw_dots(p, (double*)w, (const double*)V, ldv, j + 1, part, NBMAX, &grid));
      k_reduce_parts<<<j + 1, 256, 0, ctx->stream>>>(part, j + 1, grid, S + OFF_H, ctrl);
      k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part + (int64_t)(j + 1) * NBMAX, 1, grid, ctrl + 4, ctrl);
    } else if (MODE == kInPieces) {
      TCI_TRY(tci_heff_apply_raw(p, nullptr, w, true, kDF ? 2 : 0));
    } else if (MODE == kInNone) {
      if (p->cplx)
        TCI_TRY(tci_heff_apply_complex_raw(p, (const double*)vj, (double*)w));
      else
        TCI_TRY(tci_heff_apply_raw(p, (const double*)vj, w, false, 0));
    } else {
      TCI_TRY(tci_heff_apply_raw(p, p->lz_x64, p->lz_o64, false, 0));
      k_from_f64<A><<<NBMAX, NT, 0, ctx->stream>>>(p->lz_o64, w, n, ctrl);
    }
    if constexpr (std::is_same<A, ArithF64>::value && MODE == kInNone) {
      // short vectors: the whole step's vector work as one cluster launch
      if (reorth && n * (j + 2) <= kSmallWork) {
        const int dgks = (p->gs_mode == TCI_GS_DGKS && j + 1 <= GMAX) ? 1 : 0;
        TCI_TRY(launch_step_small(ctx, V, ldv, w, n, S, j, nsteps, tol, dgks));
        continue;
      }
    }
    if (reorth) {
      // classical Gram-Schmidt against the whole basis, repeated where the first
      // pass cancelled (DGKS); both continuations are launched, each gated
      const int dgks = (p->gs_mode == TCI_GS_DGKS && j + 1 <= GMAX) ? 1 : 0;
      // reduced-precision update terms where they pay: basis <= GMAX, long vectors
      // (below kReducedMinN the FP64 work is smaller than the extra launches)
      const bool reduced = kF32Terms && p->lz_reduced && j + 1 <= GMAX && n >= kReducedMinN;
      const double* lo1 = reduced ? S + OFF_LO : nullptr;
      if (!fused) {
        if constexpr (!kDF) {
          if (dfdots) TCI_TRY(run_dots_shadow(ctx, Vs, ldv, j + 1, (const double*)w, n, part, S + OFF_H, ctrl, ctrl + 4));
        }
        if (!dfdots) TCI_TRY(run_dots<A>(ctx, V, ldv, 0, j + 1, w, n, part, S + OFF_H, ctrl, ctrl + 4, ticket));
      }
      k_post_pass1<<<1, 1, 0, ctx->stream>>>(S, j, 1, dgks, reduced ? 1 : 0);
      // second pass taken: w -= V h, then its dots and ||w'||^2; then w -= V h'
      // with ||w||^2 in FP64, or folded into the next-vector kernel
      TCI_TRY(run_update<A>(ctx, V, ldv, 0, j + 1, S + OFF_H, w, n, part, S + OFF_H2, S + OFF_LO + LO_WN2, ctrl + 5,
                            lo1, dfdots, ticket));
      k_post_pass2<<<1, 1, 0, ctx->stream>>>(S, j, (kF32Terms && p->lz_reduced) ? 1 : 0);
      TCI_TRY(run_update<A>(ctx, V, ldv, 0, j + 1, S + OFF_H2, w, n, part, nullptr, ctrl + 3, S + OFF_LO + LO_GSLOW,
                            nullptr, false, ticket));
      // second pass skipped: w -= V h with ||w||^2
      TCI_TRY(run_update<A>(ctx, V, ldv, 0, j + 1, S + OFF_H, w, n, part, nullptr, ctrl + 3, ctrl + 6, lo1, false,
                            ticket));
    } else {
      TCI_TRY(run_dots<A>(ctx, V, ldv, j, 1, w, n, part, S + OFF_H + j, ctrl, nullptr, ticket));
      k_post_pass1<<<1, 1, 0, ctx->stream>>>(S, j, 0, 0, 0);
      const int v0 = j > 0 ? j - 1 : 0;
      TCI_TRY(run_update<A>(ctx, V, ldv, v0, j + 1 - v0, S + OFF_H, w, n, part, nullptr, ctrl + 3, ctrl, nullptr,
                            false, ticket));
    }
    k_finish_beta<<<1, 1, 0, ctx->stream>>>(S, j, nsteps, tol);
    if (j + 1 < nsteps) {
      Vt* vn = V + (int64_t)(j + 1) * ldv;
      float* vsh = Vs ? Vs + (int64_t)(j + 1) * vs_ld : nullptr;
      const ShadowOut vsn{vsh, (vsh && dfdots) ? vsh + ldv : nullptr};
      launch_next<A, MODE>(ctx, w, vn, rows, cols, pieces, Kp, p->lz_x64, S, j, reorth ? S + OFF_LO + LO_GNEXT : ctrl,
                           vsn);
      if constexpr (kF32Terms) {
        if (reorth) launch_next_corr<MODE>(ctx, V, ldv, j + 1, w, vn, rows, cols, pieces, Kp, S, j, vsn, Vs, vs_ld);
      }
    }
    TCI_CUDA(ctx, cudaGetLastError());
  }
  k_tridiag_lowest<<<1, kTriP, 0, ctx->stream>>>(S);
  if (x) k_ritz<A><<<NBMAX, NT, 0, ctx->stream>>>(V, ldv, S, x, n);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

}  // namespace

namespace {
// Point argument `idx` (a pointer; the kernel takes `nargs` arguments) of the
// graph's kernel node `node` at `value` in the instantiated graph; the other
// arguments keep their captured values.
tci_status graph_set_ptr_arg(tci_context ctx, tci_graph& g, int node, int nargs, int idx, const void* value) {
  cudaKernelNodeParams kp;
  TCI_CUDA(ctx, cudaGraphKernelNodeGetParams(g.nodes[node], &kp));
  if (!kp.kernelParams) return tci_fail(ctx, TCI_ERR_CUDA, "lanczos graph: kernel node without parameters");
  void* args[16];
  for (int i = 0; i < nargs; ++i) args[i] = kp.kernelParams[i];
  const void* v = value;
  args[idx] = (void*)&v;
  kp.kernelParams = args;
  kp.extra = nullptr;
  TCI_CUDA(ctx, cudaGraphExecKernelNodeSetParams(g.exec, g.nodes[node], &kp));
  return TCI_OK;
}

struct SolveArgs {
  tci_heff_plan p;
  const double* psi;
  int nsteps, reorth;
  double* x;
  double tol;
  int arith;
  bool split;
  float* Vs;
  bool dfdots;
};

// One solve's launches on p->ctx->stream (the body a graph captures).
tci_status solve_body(void* a) {
  const SolveArgs& s = *(const SolveArgs*)a;
  if (s.arith == TCI_LANCZOS_DF32) {
    if (s.split) return lanczos_run<ArithDF, kInPieces>(s.p, s.psi, s.nsteps, s.reorth, s.x, s.tol, nullptr, false);
    return lanczos_run<ArithDF, kInF64>(s.p, s.psi, s.nsteps, s.reorth, s.x, s.tol, nullptr, false);
  }
  if (s.split) return lanczos_run<ArithF64, kInPieces>(s.p, s.psi, s.nsteps, s.reorth, s.x, s.tol, s.Vs, s.dfdots);
  return lanczos_run<ArithF64, kInNone>(s.p, s.psi, s.nsteps, s.reorth, s.x, s.tol, nullptr, false);
}
}  // namespace

extern "C" tci_status tci_lanczos(tci_heff_plan p, tci_tensor psi0, int nsteps, int reorth, double* ritz, double* alpha,
                                  double* beta, int* steps_done, tci_tensor x) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "lanczos: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "lanczos");
  if (nsteps < 1 || nsteps > MAXM) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "lanczos: nsteps must be in 1..%d", MAXM);
  if (!ritz) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "lanczos: NULL ritz output");
  const tci_dtype vdt = p->cplx ? TCI_C128 : TCI_F64;
  const int64_t d = p->cplx ? p->cd : 2;
  auto check = [&](tci_tensor t, const char* what) -> tci_status {
    if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "lanczos: invalid %s", what);
    if (t->dtype != vdt) return tci_fail(ctx, TCI_ERR_DTYPE, "lanczos: %s must be %s", what, p->cplx ? "C128" : "F64");
    if (t->order != 4 || t->shape[0] != p->chiL || t->shape[1] != d || t->shape[2] != d || t->shape[3] != p->chiR ||
        !tci_is_rowmajor(t))
      return tci_fail(ctx, TCI_ERR_SHAPE, "lanczos: %s must be row-major [chiL,d,d,chiR]", what);
    return TCI_OK;
  };
  TCI_TRY(check(psi0, "psi0"));
  if (x) TCI_TRY(check(x, "x"));
  if (p->cplx && p->vec_arith == TCI_LANCZOS_DF32)
    return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "lanczos: complex plans run FP64 vectors only");
  const int64_t n = p->cplx ? 2 * p->chiL * d * d * p->chiR : p->chiL * 4 * p->chiR;
  const int64_t ldv = (n + 31) / 32 * 32;
  if (p->lz_cap < nsteps + 1) {
    cudaStreamSynchronize(ctx->stream);
    tci_dev_free(p->lz_V);
    p->lz_V = nullptr;
    p->lz_cap = 0;
    TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * ldv * (nsteps + 1), (void**)&p->lz_V));
    p->lz_cap = nsteps + 1;
  }
  if (!p->lz_w) TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * n, (void**)&p->lz_w));
  if (!p->lz_scal) TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * NSCAL, (void**)&p->lz_scal));
  if (!p->lz_part) TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * (int64_t)NBMAX * (MAXM + 1), (void**)&p->lz_part));
  double* S = p->lz_scal;
  double* ctrl = S + OFF_CTRL;
  const double tol = 1e-12;
  const int arith = p->vec_arith == TCI_LANCZOS_DF32 ? TCI_LANCZOS_DF32 : TCI_LANCZOS_F64;
  const bool split = p->prec != TCI_PREC_NATIVE;
  vs.info = arith == TCI_LANCZOS_DF32 ? "double-float vectors" : "FP64 vectors";
  const double* psi = (const double*)psi0->data;
  double* xd = x ? (double*)x->data : nullptr;
  // the basis copy (split plans, FP64 vectors, re-orthogonalised, dots not
  // fused into GEMM2): its FP32 planes serve the pass-3 correction, and with
  // shadow (the opt-in double-float dots) its lo planes too
  const bool copy = split && arith == TCI_LANCZOS_F64 && !p->cplx && reorth && !p->lz_fuse;
  const bool shadow = copy && p->lz_shadow;
  const int vs_planes = copy ? p->lz_cap * (shadow ? 2 : 1) : 0;   // FP32 planes of ldv elements
  if (copy && p->lz_vs_cap < vs_planes) {
    cudaStreamSynchronize(ctx->stream);
    tci_dev_free(p->lz_Vs);
    p->lz_Vs = nullptr;
    p->lz_vs_cap = 0;
    TCI_TRY(tci_dev_alloc(ctx, sizeof(float) * ldv * vs_planes, &p->lz_Vs));
    p->lz_vs_cap = vs_planes;
  }
  SolveArgs sa{p, psi, nsteps, reorth, xd, tol, arith, split, copy ? (float*)p->lz_Vs : nullptr, shadow};
  bool done = false;
  p->lz_last_graph = 0;
  if (!p->cplx && p->lz_graphs) {
    // eager on the first call with a key, captured on the second, replayed after;
    // psi0 and x are not part of the key: the three kernel nodes that read psi0
    // or write x get the call's pointers before every replay
    const std::vector<int64_t> key = {xd != nullptr, nsteps, reorth, arith, p->gs_mode, p->lz_reduced, p->lz_fuse,
                                      shadow, copy, (int64_t)(uintptr_t)p->lz_Vs, p->products,
                                      p->chunk_k,
                                      p->xchunk_k, p->raster, p->ww_na, (int64_t)(uintptr_t)p->lz_V,
                                      (int64_t)ctx->wait_limit_ns};
    const bool df = arith == TCI_LANCZOS_DF32;
    const void* start_fn = split ? (df ? (const void*)k_start<ArithDF, kInPieces> : (const void*)k_start<ArithF64, kInPieces>)
                                 : (df ? (const void*)k_start<ArithDF, kInF64> : (const void*)k_start<ArithF64, kInNone>);
    std::vector<const void*> io = {(const void*)k_sumsq, start_fn};
    if (xd) io.push_back(df ? (const void*)k_ritz<ArithDF> : (const void*)k_ritz<ArithF64>);
    if (!(p->lz_graph.exec && key == p->lz_graph_key) && key == p->lz_last_key) {
      tci_graph_destroy(&p->lz_graph);
      p->lz_graph_key.clear();
      if (tci_graph_capture(ctx, &p->lz_graph, solve_body, &sa, io) == TCI_OK) {
        p->lz_graph_key = key;
      } else {   // run eagerly from now on
        tci_graph_destroy(&p->lz_graph);
        cudaGetLastError();
        p->lz_graphs = 0;
      }
    }
    if (p->lz_graph.exec && key == p->lz_graph_key) {
      // k_sumsq(psi0, n, part), k_start(psi0, ...), k_ritz(V, ldv, S, x, n)
      TCI_TRY(graph_set_ptr_arg(ctx, p->lz_graph, 0, 3, 0, psi));
      TCI_TRY(graph_set_ptr_arg(ctx, p->lz_graph, 1, 9, 0, psi));
      if (xd) TCI_TRY(graph_set_ptr_arg(ctx, p->lz_graph, 2, 5, 3, xd));
      TCI_CUDA(ctx, cudaGraphLaunch(p->lz_graph.exec, ctx->stream));
      done = true;
      p->lz_last_graph = 1;
      ++p->lz_graph_launches;
    }
    p->lz_last_key = key;
  }
  if (!done) TCI_TRY(solve_body(&sa));
  TCI_CUDA(ctx, cudaMemcpyAsync(ctx->h_scalars, ctrl, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<double> ab(2 * MAXM), cnt(4);
  TCI_CUDA(ctx, cudaMemcpyAsync(ab.data(), S, 2 * MAXM * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  TCI_CUDA(ctx, cudaMemcpyAsync(cnt.data(), S + OFF_LO + LO_N1, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->stream));
  static_assert(LO_N3 == LO_N1 + 1 && LO_N2 == LO_N1 + 3, "counter layout");
  TCI_TRY(tci_synchronize(ctx));
  const int k = (int)ctx->h_scalars[1];
  *ritz = ctx->h_scalars[2];
  p->lz_stats[0] = k;
  p->lz_stats[1] = reorth ? (int)ctx->h_scalars[7] : 0;
  p->lz_stats[2] = (int)cnt[0];
  p->lz_stats[3] = (int)cnt[3];
  p->lz_stats[4] = (int)cnt[1];
  if (ctx->verbose > 0 && reorth)
    vs.info += " second_gs_passes=" + std::to_string(p->lz_stats[1]) + " f32_term_passes=" +
               std::to_string(p->lz_stats[2]) + " df_term_passes=" + std::to_string(p->lz_stats[3]) +
               " fused_pass3=" + std::to_string(p->lz_stats[4]);
  if (steps_done) *steps_done = k;
  for (int i = 0; i < nsteps; ++i) {
    if (alpha) alpha[i] = i < k ? ab[OFF_ALPHA + i] : 0.0;
    if (beta) beta[i] = i < k ? ab[OFF_BETA + i] : 0.0;
  }
  return TCI_OK;
}

extern "C" tci_status tci_heff_set_lanczos_arith(tci_heff_plan p, tci_lanczos_arith arith) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "set_lanczos_arith: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  if (arith != TCI_LANCZOS_AUTO && arith != TCI_LANCZOS_F64 && arith != TCI_LANCZOS_DF32)
    return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "set_lanczos_arith: unknown arithmetic %d", (int)arith);
  p->vec_arith = (int)arith;
  return TCI_OK;
}

extern "C" tci_status tci_heff_set_gram_schmidt(tci_heff_plan p, tci_gram_schmidt mode) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "set_gram_schmidt: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  if (mode != TCI_GS_DGKS && mode != TCI_GS_TWICE)
    return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "set_gram_schmidt: unknown mode %d", (int)mode);
  p->gs_mode = (int)mode;
  return TCI_OK;
}

extern "C" tci_status tci_heff_lanczos_stats(tci_heff_plan p, int* stats) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "lanczos_stats: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  if (!stats) return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "lanczos_stats: NULL stats");
  for (int i = 0; i < 5; ++i) stats[i] = p->lz_stats[i];
  return TCI_OK;
}

extern "C" tci_status tci_heff_lanczos_graph_info(tci_heff_plan p, int64_t* info) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "lanczos_graph_info: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  if (!info) return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "lanczos_graph_info: NULL info");
  info[0] = p->lz_graphs;
  info[1] = p->lz_last_graph;
  info[2] = p->lz_graph_launches;
  return TCI_OK;
}

extern "C" tci_status tci_heff_set_lanczos_graphs(tci_heff_plan p, int enable) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "set_lanczos_graphs: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  p->lz_graphs = enable ? 1 : 0;
  if (!enable) {
    cudaStreamSynchronize(p->ctx->stream);
    tci_graph_destroy(&p->lz_graph);
    p->lz_graph_key.clear();
    p->lz_last_key.clear();
  }
  return TCI_OK;
}

extern "C" tci_status tci_heff_set_lanczos_fused_dots(tci_heff_plan p, int enable) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "set_lanczos_fused_dots: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  p->lz_fuse = enable ? 1 : 0;
  return TCI_OK;
}

extern "C" tci_status tci_heff_set_lanczos_shadow_dots(tci_heff_plan p, int enable) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "set_lanczos_shadow_dots: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  p->lz_shadow = enable ? 1 : 0;
  return TCI_OK;
}

extern "C" tci_status tci_heff_set_lanczos_reduced_terms(tci_heff_plan p, int enable) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "set_lanczos_reduced_terms: invalid plan");
  TCI_CHECK_CTX(p->ctx);
  p->lz_reduced = enable ? 1 : 0;
  return TCI_OK;
}
