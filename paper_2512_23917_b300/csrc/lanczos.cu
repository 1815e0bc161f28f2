// Lanczos ground-state solve of H_eff on the device (textbook: Golub &
// Van Loan Sec. 10.1; classical Gram-Schmidt applied twice for full
// re-orthogonalisation; Sturm-sequence bisection, Sec. 8.4, and inverse
// iteration for the tridiagonal eigenpair).
//
// Two kinds of vector arithmetic:
//   FP64         every dot and update in FP64 (default for the FP64 matvec);
//   double-float vectors stored as FP32 pairs hi + lo (~48 significant bits;
//                default for the split-BF16 matvec, whose own error is ~1e-7).
//                B300 runs FP64 FMAs at ~1/64 of its FP32 rate: FP64 dots
//                over HBM-resident vectors are FP64-pipe bound, double-float
//                ones stay HBM bound.  This variant also fuses the passes:
//                CGS pass 1 (whose coefficient for v_j is alpha_j and whose
//                update subsumes the three-term recurrence), pass 2's update
//                with pass 2's dots, the last update with ||w||^2, and the
//                normalisation of v_{j+1} with the operand split of the next
//                matvec.
//
// All scalars (alpha, beta, re-orthogonalisation coefficients, stop flag,
// step count, Ritz coefficients) stay in device memory; the host enqueues
// the whole sequence and reads back once at the end.  Reductions are
// deterministic: a fixed grid, a fixed per-thread order and an in-order sum
// of the block partials.
#include <cuda_bf16.h>

#include "heff_plan.cuh"

namespace {

constexpr int NB = 1184;         // 8 x 148 SMs: blocks of every reduction (64 warps per SM)
constexpr int NT = 256;
constexpr int MAXM = 256;
// device scalar layout (doubles)
constexpr int OFF_ALPHA = 0;
constexpr int OFF_BETA = MAXM;
constexpr int OFF_H = 2 * MAXM;          // MAXM + 1 entries
constexpr int OFF_CTRL = 3 * MAXM + 8;   // [0] stop flag, [1] steps done, [2] theta, [3] sumsq
constexpr int OFF_Y = 3 * MAXM + 16;
constexpr int OFF_H2 = 4 * MAXM + 32;    // MAXM + 1 entries (double-float path: pass-2 coefficients)
constexpr int NSCAL = 5 * MAXM + 64;
constexpr int DF_GMAX = 24;              // basis vectors per fused double-float pass

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// part[v*NB + block] = sum over this block's slice of V_v[i] * w[i], v < nv.
// Each thread walks two grid-stride elements per iteration (independent FP64
// chains); the per-thread order is fixed, so the result is deterministic.
template <int G>
__global__ void __launch_bounds__(NT) k_mdot(const double* __restrict__ V, int64_t ldv, int v0, int nv,
                                             const double* __restrict__ w, int64_t n, double* __restrict__ part,
                                             const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  __shared__ double sh[NT / 32][G];
  double acc[G], acc2[G];
#pragma unroll
  for (int g = 0; g < G; ++g) acc[g] = acc2[g] = 0.0;
  const int64_t stride = (int64_t)NB * NT;
  int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x;
  for (; i + stride < n; i += 2 * stride) {
    const double wi = w[i], wj = w[i + stride];
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < nv) {
        const double* vg = V + (int64_t)(v0 + g) * ldv;
        acc[g] = fma(vg[i], wi, acc[g]);
        acc2[g] = fma(vg[i + stride], wj, acc2[g]);
      }
  }
  if (i < n) {
    const double wi = w[i];
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < nv) acc[g] = fma(V[(int64_t)(v0 + g) * ldv + i], wi, acc[g]);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    double s = warp_sum(acc[g] + acc2[g]);
    if (lane == 0) sh[wid][g] = s;
  }
  __syncthreads();
  if (threadIdx.x < G && threadIdx.x < nv) {
    double s = 0.0;
    for (int k = 0; k < NT / 32; ++k) s += sh[k][threadIdx.x];
    part[(int64_t)(v0 + threadIdx.x) * NB + blockIdx.x] = s;
  }
}

// out[v] = sum_b part[v*NB + b] in order; one block per vector.
__global__ void k_reduce_parts(const double* __restrict__ part, int nv, double* __restrict__ out,
                               const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  const int v = blockIdx.x;
  if (v >= nv) return;
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < NB; b += blockDim.x) s += part[(int64_t)v * NB + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    out[v] = r;
  }
}

// w -= sum_{v<nv} c[v] V_v   (two elements per thread per iteration)
template <int G>
__global__ void __launch_bounds__(NT) k_mupdate(const double* __restrict__ V, int64_t ldv, int v0, int nv,
                                                const double* __restrict__ c, double* __restrict__ w, int64_t n,
                                                const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  double cc[G];
#pragma unroll
  for (int g = 0; g < G; ++g) cc[g] = g < nv ? c[v0 + g] : 0.0;
  const int64_t stride = (int64_t)NB * NT;
  int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x;
  for (; i + stride < n; i += 2 * stride) {
    double s = 0.0, t = 0.0;
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < nv) {
        const double* vg = V + (int64_t)(v0 + g) * ldv;
        s = fma(cc[g], vg[i], s);
        t = fma(cc[g], vg[i + stride], t);
      }
    w[i] -= s;
    w[i + stride] -= t;
  }
  if (i < n) {
    double s = 0.0;
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < nv) s = fma(cc[g], V[(int64_t)(v0 + g) * ldv + i], s);
    w[i] -= s;
  }
}

// w = w - alpha_j v_j - beta_{j-1} v_{j-1}
__global__ void __launch_bounds__(NT) k_three_term(double* __restrict__ w, const double* __restrict__ vj,
                                                   const double* __restrict__ vjm1, int64_t n,
                                                   const double* __restrict__ scal, int j) {
  if (scal[OFF_CTRL] != 0.0) return;
  const double a = scal[OFF_ALPHA + j];
  const double b = j > 0 ? scal[OFF_BETA + j - 1] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) {
    double x = w[i] - a * vj[i];
    if (j > 0) x -= b * vjm1[i];
    w[i] = x;
  }
}

__global__ void __launch_bounds__(NT) k_sumsq(const double* __restrict__ w, int64_t n, double* __restrict__ part,
                                              const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  __shared__ double sh[NT / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) acc = fma(w[i], w[i], acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < NT / 32; ++k) s += sh[k];
    part[blockIdx.x] = s;
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

// v_{j+1} = w / beta_j (unless stopped)
__global__ void __launch_bounds__(NT) k_next_vec(const double* __restrict__ w, double* __restrict__ vn, int64_t n,
                                                 const double* __restrict__ scal, int j) {
  if (scal[OFF_CTRL] != 0.0) return;
  const double inv = 1.0 / scal[OFF_BETA + j];
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) vn[i] = w[i] * inv;
}

// v_0 = psi / ||psi||  (sumsq partial sums already in part[0..NB))
__global__ void __launch_bounds__(NT) k_start_vec(const double* __restrict__ psi, double* __restrict__ v0, int64_t n,
                                                  const double* __restrict__ scal) {
  const double inv = 1.0 / sqrt(scal[OFF_CTRL + 3]);
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) v0[i] = psi[i] * inv;
}

// x = sum_{j<k} y_j v_j
__global__ void __launch_bounds__(NT) k_ritz_vec(const double* __restrict__ V, int64_t ldv,
                                                 const double* __restrict__ scal, double* __restrict__ x, int64_t n) {
  const int k = (int)scal[OFF_CTRL + 1];
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s = fma(scal[OFF_Y + j], V[(int64_t)j * ldv + i], s);
    x[i] = s;
  }
}

__device__ int sturm_count(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < m; ++i) {
    if (i == 0) {
      q = a[0] - x;
    } else {
      if (q == 0.0) q = -2.2250738585072014e-308;
      q = a[i] - x - b[i - 1] * b[i - 1] / q;
    }
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// K7: lowest eigenpair of T_k = tridiag(beta, alpha, beta) in one CTA:
// multisection on the Sturm count (each of NT threads tests one point per
// round), then inverse iteration with Gaussian elimination with partial
// pivoting on T - sigma I.
__global__ void __launch_bounds__(NT) k_tridiag_lowest(double* scal) {
  __shared__ double a[MAXM], b[MAXM];
  __shared__ double lo, hi;
  __shared__ int first;
  const int m = (int)scal[OFF_CTRL + 1];
  if (m <= 0) return;
  for (int i = threadIdx.x; i < m; i += NT) {
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
  for (int round = 0; round < 64; ++round) {
    const double l = lo, h = hi;
    const double x = l + (h - l) * (double)(threadIdx.x + 1) / (double)(NT + 1);
    if (threadIdx.x == 0) first = NT;
    __syncthreads();
    const bool hit = x > l && x < h && sturm_count(a, b, m, x) >= 1;
    if (hit) atomicMin(&first, (int)threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int f = first;
      double nl = l, nh = h;
      if (f < NT) {
        nh = l + (h - l) * (double)(f + 1) / (double)(NT + 1);
        if (f > 0) nl = l + (h - l) * (double)f / (double)(NT + 1);
      } else {
        nl = l + (h - l) * (double)NT / (double)(NT + 1);
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

__global__ void k_init_scal(double* scal) {
  for (int i = threadIdx.x; i < NSCAL; i += blockDim.x) scal[i] = 0.0;
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

// (h, l) += x * y
__device__ __forceinline__ void df_acc(float2 x, float2 y, float& h, float& l) {
  float p, t, s, err;
  df_prod(x, y, p, t);
  df_two_sum(h, p, s, err);
  h = s;
  l = __fadd_rn(l, __fadd_rn(err, t));
}

// (h, l) -= x * y
__device__ __forceinline__ void df_sub(float2 x, float2 y, float& h, float& l) {
  float p, t, s, err;
  df_prod(x, y, p, t);
  df_two_sum(h, -p, s, err);
  h = s;
  l = __fadd_rn(l, __fsub_rn(err, t));
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

// Per-block partial sums of G double-float accumulators (fixed order):
// part[g*NB + blockIdx.x] for g < nv.
template <int G>
__device__ __forceinline__ void df_block_partials(const float (&h)[G], const float (&l)[G], int nv, double* part) {
  __shared__ double sh[NT / 32][G];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (g < nv) {
      const double s = warp_sum((double)h[g] + (double)l[g]);
      if (lane == 0) sh[wid][g] = s;
    }
  __syncthreads();
  if (threadIdx.x < G && threadIdx.x < nv) {
    double s = 0.0;
    for (int k = 0; k < NT / 32; ++k) s += sh[k][threadIdx.x];
    part[(int64_t)threadIdx.x * NB + blockIdx.x] = s;
  }
}

// part[(v0+g)*NB + block] = partial <V_{v0+g}, w>, g < nv <= G
template <int G>
__global__ void __launch_bounds__(NT) k_df_dots(const float2* __restrict__ V, int64_t ldv, int v0, int nv,
                                                const float2* __restrict__ w, int64_t n, double* __restrict__ part,
                                                const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  float h[G], l[G];
#pragma unroll
  for (int g = 0; g < G; ++g) h[g] = l[g] = 0.f;
  const float2* Vb = V + (int64_t)v0 * ldv;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) {
    const float2 x = w[i];
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < nv) df_acc(Vb[(int64_t)g * ldv + i], x, h[g], l[g]);
  }
  df_block_partials<G>(h, l, nv, part + (int64_t)v0 * NB);
}

// w -= sum_{g<nv} coef[v0+g] V_{v0+g}; then optionally the partial dots of
// the new w with the same vectors (part rows v0..) and of ||w||^2 (part_sq).
template <int G, bool DOTS, bool SUMSQ>
__global__ void __launch_bounds__(NT) k_df_update(const float2* __restrict__ V, int64_t ldv, int v0, int nv,
                                                  const double* __restrict__ coef, float2* __restrict__ w, int64_t n,
                                                  double* __restrict__ part, double* __restrict__ part_sq,
                                                  const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  __shared__ float2 cs[G];
  if (threadIdx.x < G) cs[threadIdx.x] = threadIdx.x < nv ? df_from_double(coef[v0 + threadIdx.x]) : make_float2(0.f, 0.f);
  __syncthreads();
  constexpr int GD = DOTS ? G : 1;
  float dh[GD], dl[GD];
#pragma unroll
  for (int g = 0; g < GD; ++g) dh[g] = dl[g] = 0.f;
  float qh = 0.f, ql = 0.f;
  const float2* Vb = V + (int64_t)v0 * ldv;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) {
    float2 v[G];
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < nv) v[g] = Vb[(int64_t)g * ldv + i];
    const float2 x = w[i];
    float h = x.x, l = x.y;
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < nv) df_sub(cs[g], v[g], h, l);
    const float2 y = df_norm(h, l);
    w[i] = y;
    if (DOTS) {
#pragma unroll
      for (int g = 0; g < GD; ++g)
        if (g < nv) df_acc(v[g], y, dh[g], dl[g]);
    }
    if (SUMSQ) df_acc(y, y, qh, ql);
  }
  if (DOTS) df_block_partials<GD>(dh, dl, nv, part + (int64_t)v0 * NB);
  if (SUMSQ) {
    float qa[1] = {qh}, qb[1] = {ql};
    if (DOTS) __syncthreads();
    df_block_partials<1>(qa, qb, 1, part_sq);
  }
}

// alpha_j = <v_j, H v_j> (the pass-1 coefficient of v_j); without
// re-orthogonalisation the update coefficients are (beta_{j-1}, alpha_j).
__global__ void k_df_post_pass1(double* scal, int j, int reorth) {
  if (scal[OFF_CTRL] != 0.0) return;
  scal[OFF_ALPHA + j] = scal[OFF_H + j];
  if (!reorth && j > 0) scal[OFF_H + j - 1] = scal[OFF_BETA + j - 1];
}

// Store a new basis vector y (already normalised) at element (r, k) and the
// matvec's input: bfloat16 pieces of fl32(y) = y.hi (K-major [3][rows][Kp],
// zero in k >= cols) or, for the FP64 matvec, y as FP64.
template <bool PIECES>
__device__ __forceinline__ void df_emit(float2 y, int64_t i, int64_t r, int64_t k, float2* vn, __nv_bfloat16* pieces,
                                        int64_t Kp, int64_t plane, double* x64) {
  vn[i] = y;
  if (PIECES) split3_store(pieces + r * Kp + k, plane, y.x);
  else x64[i] = (double)y.x + (double)y.y;
}

// v_{j+1} = w / beta_j (unless stopped), one row (r) per block iteration.
template <bool PIECES>
__global__ void __launch_bounds__(NT) k_df_next(const float2* __restrict__ w, float2* __restrict__ vn, int64_t rows,
                                                int64_t cols, __nv_bfloat16* __restrict__ pieces, int64_t Kp,
                                                double* __restrict__ x64, const double* __restrict__ scal, int j) {
  if (scal[OFF_CTRL] != 0.0) return;
  const float2 c = df_from_double(1.0 / scal[OFF_BETA + j]);
  const int64_t plane = rows * Kp;
  const int64_t kend = PIECES ? Kp : cols;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t k = threadIdx.x; k < kend; k += NT) {
      if (k < cols) {
        const int64_t i = r * cols + k;
        float p, t;
        df_prod(w[i], c, p, t);
        df_emit<PIECES>(df_norm(p, t), i, r, k, vn, pieces, Kp, plane, x64);
      } else {
        split3_store(pieces + r * Kp + k, plane, 0.f);
      }
    }
}

// v_0 = psi / ||psi|| (FP64 sum of squares already in scal[OFF_CTRL + 3])
template <bool PIECES>
__global__ void __launch_bounds__(NT) k_df_start(const double* __restrict__ psi, float2* __restrict__ v0, int64_t rows,
                                                 int64_t cols, __nv_bfloat16* __restrict__ pieces, int64_t Kp,
                                                 double* __restrict__ x64, const double* __restrict__ scal) {
  const double inv = 1.0 / sqrt(scal[OFF_CTRL + 3]);
  const int64_t plane = rows * Kp;
  const int64_t kend = PIECES ? Kp : cols;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t k = threadIdx.x; k < kend; k += NT) {
      if (k < cols) {
        const int64_t i = r * cols + k;
        df_emit<PIECES>(df_from_double(psi[i] * inv), i, r, k, v0, pieces, Kp, plane, x64);
      } else {
        split3_store(pieces + r * Kp + k, plane, 0.f);
      }
    }
}

__global__ void __launch_bounds__(NT) k_f64_to_df(const double* __restrict__ x, float2* __restrict__ y, int64_t n,
                                                  const double* __restrict__ ctrl) {
  if (ctrl[0] != 0.0) return;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) y[i] = df_from_double(x[i]);
}

// x = sum_{j<k} y_j v_j, accumulated in double-float, stored as FP64
__global__ void __launch_bounds__(NT) k_df_ritz(const float2* __restrict__ V, int64_t ldv,
                                                const double* __restrict__ scal, double* __restrict__ x, int64_t n) {
  __shared__ float2 ys[MAXM];
  const int k = (int)scal[OFF_CTRL + 1];
  for (int j = threadIdx.x; j < k; j += NT) ys[j] = df_from_double(scal[OFF_Y + j]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)NB * NT) {
    float h = 0.f, l = 0.f;
    for (int j = 0; j < k; ++j) df_acc(ys[j], V[(int64_t)j * ldv + i], h, l);
    x[i] = (double)h + (double)l;
  }
}

}  // namespace

static tci_status mdot(tci_context ctx, const double* V, int64_t ldv, int nv, const double* w, int64_t n, double* part,
                       double* out, const double* ctrl) {
  for (int v0 = 0; v0 < nv; v0 += 8) {
    const int g = nv - v0 < 8 ? nv - v0 : 8;
    k_mdot<8><<<NB, NT, 0, ctx->stream>>>(V, ldv, v0, g, w, n, part, ctrl);
  }
  k_reduce_parts<<<nv, 256, 0, ctx->stream>>>(part, nv, out, ctrl);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

static tci_status mupdate(tci_context ctx, const double* V, int64_t ldv, int nv, const double* c, double* w, int64_t n,
                          const double* ctrl) {
  for (int v0 = 0; v0 < nv; v0 += 8) {
    const int g = nv - v0 < 8 ? nv - v0 : 8;
    k_mupdate<8><<<NB, NT, 0, ctx->stream>>>(V, ldv, v0, g, c, w, n, ctrl);
  }
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

// ---------------------------------------------------------------- double-float host helpers
template <int G>
static void df_dots_launch(tci_context ctx, const float2* V, int64_t ldv, int v0, int nv, const float2* w, int64_t n,
                           double* part, const double* ctrl) {
  k_df_dots<G><<<NB, NT, 0, ctx->stream>>>(V, ldv, v0, nv, w, n, part, ctrl);
}

// out[0..nv) = <V_v, w>
static tci_status df_dots(tci_context ctx, const float2* V, int64_t ldv, int v0, int nv, const float2* w, int64_t n,
                          double* part, double* out, const double* ctrl) {
  for (int g0 = 0; g0 < nv; g0 += DF_GMAX) {
    const int g = nv - g0 < DF_GMAX ? nv - g0 : DF_GMAX;
    if (g <= 8) df_dots_launch<8>(ctx, V, ldv, v0 + g0, g, w, n, part, ctrl);
    else if (g <= 16) df_dots_launch<16>(ctx, V, ldv, v0 + g0, g, w, n, part, ctrl);
    else df_dots_launch<DF_GMAX>(ctx, V, ldv, v0 + g0, g, w, n, part, ctrl);
  }
  k_reduce_parts<<<nv, 256, 0, ctx->stream>>>(part + (int64_t)v0 * NB, nv, out, ctrl);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

template <bool DOTS, bool SUMSQ>
static void df_update_launch(tci_context ctx, const float2* V, int64_t ldv, int v0, int nv, const double* coef,
                             float2* w, int64_t n, double* part, double* part_sq, const double* ctrl) {
  if (nv <= 8)
    k_df_update<8, DOTS, SUMSQ><<<NB, NT, 0, ctx->stream>>>(V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl);
  else if (nv <= 16)
    k_df_update<16, DOTS, SUMSQ><<<NB, NT, 0, ctx->stream>>>(V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl);
  else
    k_df_update<DF_GMAX, DOTS, SUMSQ><<<NB, NT, 0, ctx->stream>>>(V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl);
}

// w -= sum_{v0 <= v < v0+nv} coef[v] V_v; then dots_out[0..nv) = <V_v, w>
// (when dots_out) and *sumsq_out = ||w||^2 (when sumsq_out).  One fused
// pass for nv <= DF_GMAX; larger sets update group by group and take the
// dots in a separate pass.
static tci_status df_update(tci_context ctx, const float2* V, int64_t ldv, int v0, int nv, const double* coef,
                            float2* w, int64_t n, double* part, double* dots_out, double* sumsq_out,
                            const double* ctrl) {
  double* part_sq = part + (int64_t)MAXM * NB;
  if (nv <= DF_GMAX) {
    if (dots_out && !sumsq_out) df_update_launch<true, false>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl);
    else if (!dots_out && sumsq_out) df_update_launch<false, true>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl);
    else if (!dots_out && !sumsq_out) df_update_launch<false, false>(ctx, V, ldv, v0, nv, coef, w, n, part, part_sq, ctrl);
    else return tci_fail(ctx, TCI_ERR_INVALID_ARG, "lanczos: internal (dots and sumsq in one pass)");
    if (dots_out) k_reduce_parts<<<nv, 256, 0, ctx->stream>>>(part + (int64_t)v0 * NB, nv, dots_out, ctrl);
  } else {
    for (int g0 = 0; g0 < nv; g0 += DF_GMAX) {
      const int g = nv - g0 < DF_GMAX ? nv - g0 : DF_GMAX;
      const bool last = g0 + g == nv;
      if (last && sumsq_out) df_update_launch<false, true>(ctx, V, ldv, v0 + g0, g, coef, w, n, part, part_sq, ctrl);
      else df_update_launch<false, false>(ctx, V, ldv, v0 + g0, g, coef, w, n, part, part_sq, ctrl);
    }
    if (dots_out) TCI_TRY(df_dots(ctx, V, ldv, v0, nv, w, n, part, dots_out, ctrl));
  }
  if (sumsq_out) k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part_sq, 1, sumsq_out, ctrl);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

// The double-float Lanczos iteration (same recurrence as the FP64 one; see
// the file header for the fused pass structure).
static tci_status lanczos_df(tci_heff_plan p, const double* psi0, int nsteps, int reorth, double* x, double tol) {
  tci_context ctx = p->ctx;
  const int64_t n = p->chiL * 4 * p->chiR;
  const int64_t ldv = (n + 31) / 32 * 32;
  const int64_t rows = p->chiL * 4, cols = p->chiR;
  const bool split = p->prec != TCI_PREC_NATIVE;
  if (!split) {
    if (!p->lz_x64) TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * n, (void**)&p->lz_x64));
    if (!p->lz_o64) TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * n, (void**)&p->lz_o64));
  }
  double* S = p->lz_scal;
  double* ctrl = S + OFF_CTRL;
  float2* V = (float2*)p->lz_V;
  float2* w = (float2*)p->lz_w;
  double* part = p->lz_part;
  __nv_bfloat16* pieces = (__nv_bfloat16*)p->psip;
  const int Kp = (int)(split ? p->Kp1 : 0);
  const int rblocks = (int)(rows < (int64_t)NB * 8 ? rows : (int64_t)NB * 8);

  k_init_scal<<<1, 256, 0, ctx->stream>>>(S);
  k_sumsq<<<NB, NT, 0, ctx->stream>>>(psi0, n, part, ctrl);
  k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part, 1, ctrl + 3, ctrl);
  if (split) k_df_start<true><<<rblocks, NT, 0, ctx->stream>>>(psi0, V, rows, cols, pieces, Kp, nullptr, S);
  else k_df_start<false><<<rblocks, NT, 0, ctx->stream>>>(psi0, V, rows, cols, nullptr, 0, p->lz_x64, S);
  TCI_CUDA(ctx, cudaGetLastError());
  for (int j = 0; j < nsteps; ++j) {
    // w = H v_j (the matvec's input was prepared with v_j)
    if (split) {
      TCI_TRY(tci_heff_apply_raw(p, nullptr, w, true, 2));
    } else {
      TCI_TRY(tci_heff_apply_raw(p, p->lz_x64, p->lz_o64, false, 0));
      k_f64_to_df<<<NB, NT, 0, ctx->stream>>>(p->lz_o64, w, n, ctrl);
    }
    if (reorth) {
      TCI_TRY(df_dots(ctx, V, ldv, 0, j + 1, w, n, part, S + OFF_H, ctrl));
      k_df_post_pass1<<<1, 1, 0, ctx->stream>>>(S, j, 1);
      TCI_TRY(df_update(ctx, V, ldv, 0, j + 1, S + OFF_H, w, n, part, S + OFF_H2, nullptr, ctrl));
      TCI_TRY(df_update(ctx, V, ldv, 0, j + 1, S + OFF_H2, w, n, part, nullptr, ctrl + 3, ctrl));
    } else {
      TCI_TRY(df_dots(ctx, V, ldv, j, 1, w, n, part, S + OFF_H + j, ctrl));
      k_df_post_pass1<<<1, 1, 0, ctx->stream>>>(S, j, 0);
      const int v0 = j > 0 ? j - 1 : 0;
      TCI_TRY(df_update(ctx, V, ldv, v0, j + 1 - v0, S + OFF_H, w, n, part, nullptr, ctrl + 3, ctrl));
    }
    k_finish_beta<<<1, 1, 0, ctx->stream>>>(S, j, nsteps, tol);
    if (j + 1 < nsteps) {
      float2* vn = V + (int64_t)(j + 1) * ldv;
      if (split) k_df_next<true><<<rblocks, NT, 0, ctx->stream>>>(w, vn, rows, cols, pieces, Kp, nullptr, S, j);
      else k_df_next<false><<<rblocks, NT, 0, ctx->stream>>>(w, vn, rows, cols, nullptr, 0, p->lz_x64, S, j);
    }
    TCI_CUDA(ctx, cudaGetLastError());
  }
  k_tridiag_lowest<<<1, NT, 0, ctx->stream>>>(S);
  if (x) k_df_ritz<<<NB, NT, 0, ctx->stream>>>(V, ldv, S, x, n);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

// The FP64 Lanczos iteration: three-term recurrence, then (reorth) two
// classical Gram-Schmidt passes against the whole basis.
static tci_status lanczos_f64(tci_heff_plan p, const double* psi0, int nsteps, int reorth, double* x, double tol) {
  tci_context ctx = p->ctx;
  const int64_t n = p->chiL * 4 * p->chiR;
  const int64_t ldv = (n + 31) / 32 * 32;
  double* S = p->lz_scal;
  double* ctrl = S + OFF_CTRL;
  double* V = p->lz_V;
  double* w = p->lz_w;
  double* part = p->lz_part;
  k_init_scal<<<1, 256, 0, ctx->stream>>>(S);
  // v0 = psi0 / ||psi0||
  k_sumsq<<<NB, NT, 0, ctx->stream>>>(psi0, n, part, ctrl);
  k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part, 1, ctrl + 3, ctrl);
  k_start_vec<<<NB, NT, 0, ctx->stream>>>(psi0, V, n, S);
  TCI_CUDA(ctx, cudaGetLastError());
  for (int j = 0; j < nsteps; ++j) {
    double* vj = V + (int64_t)j * ldv;
    TCI_TRY(tci_heff_apply_raw(p, vj, w, false));   // FP64 out
    // alpha_j = <v_j, w>
    TCI_TRY(mdot(ctx, vj, ldv, 1, w, n, part, S + OFF_ALPHA + j, ctrl));
    k_three_term<<<NB, NT, 0, ctx->stream>>>(w, vj, j > 0 ? V + (int64_t)(j - 1) * ldv : vj, n, S, j);
    if (reorth) {
      for (int pass = 0; pass < 2; ++pass) {
        TCI_TRY(mdot(ctx, V, ldv, j + 1, w, n, part, S + OFF_H, ctrl));
        TCI_TRY(mupdate(ctx, V, ldv, j + 1, S + OFF_H, w, n, ctrl));
      }
    }
    k_sumsq<<<NB, NT, 0, ctx->stream>>>(w, n, part, ctrl);
    k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part, 1, ctrl + 3, ctrl);
    k_finish_beta<<<1, 1, 0, ctx->stream>>>(S, j, nsteps, tol);
    if (j + 1 < nsteps) k_next_vec<<<NB, NT, 0, ctx->stream>>>(w, V + (int64_t)(j + 1) * ldv, n, S, j);
    TCI_CUDA(ctx, cudaGetLastError());
  }
  k_tridiag_lowest<<<1, NT, 0, ctx->stream>>>(S);
  if (x) k_ritz_vec<<<NB, NT, 0, ctx->stream>>>(V, ldv, S, x, n);
  TCI_CUDA(ctx, cudaGetLastError());
  return TCI_OK;
}

extern "C" tci_status tci_lanczos(tci_heff_plan p, tci_tensor psi0, int nsteps, int reorth, double* ritz, double* alpha,
                                  double* beta, int* steps_done, tci_tensor x) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "lanczos: invalid plan");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "lanczos");
  if (nsteps < 1 || nsteps > MAXM) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "lanczos: nsteps must be in 1..%d", MAXM);
  if (!ritz) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "lanczos: NULL ritz output");
  auto check = [&](tci_tensor t, const char* what) -> tci_status {
    if (!tci_ten_ok(t)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "lanczos: invalid %s", what);
    if (t->dtype != TCI_F64) return tci_fail(ctx, TCI_ERR_DTYPE, "lanczos: %s must be F64", what);
    if (t->order != 4 || t->shape[0] != p->chiL || t->shape[1] != 2 || t->shape[2] != 2 || t->shape[3] != p->chiR ||
        !tci_is_rowmajor(t))
      return tci_fail(ctx, TCI_ERR_SHAPE, "lanczos: %s must be row-major [chiL,2,2,chiR]", what);
    return TCI_OK;
  };
  TCI_TRY(check(psi0, "psi0"));
  if (x) TCI_TRY(check(x, "x"));
  const int64_t n = p->chiL * 4 * p->chiR;
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
  if (!p->lz_part) TCI_TRY(tci_dev_alloc(ctx, sizeof(double) * (int64_t)NB * (MAXM + 1), (void**)&p->lz_part));
  double* S = p->lz_scal;
  double* ctrl = S + OFF_CTRL;
  const double tol = 1e-12;
  int arith = p->vec_arith;
  if (arith == TCI_LANCZOS_AUTO) arith = p->prec == TCI_PREC_NATIVE ? TCI_LANCZOS_F64 : TCI_LANCZOS_DF32;
  vs.info = arith == TCI_LANCZOS_DF32 ? "double-float vectors" : "FP64 vectors";
  const double* psi = (const double*)psi0->data;
  double* xd = x ? (double*)x->data : nullptr;
  if (arith == TCI_LANCZOS_DF32) TCI_TRY(lanczos_df(p, psi, nsteps, reorth, xd, tol));
  else TCI_TRY(lanczos_f64(p, psi, nsteps, reorth, xd, tol));
  TCI_CUDA(ctx, cudaMemcpyAsync(ctx->h_scalars, ctrl, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<double> ab(2 * MAXM);
  TCI_CUDA(ctx, cudaMemcpyAsync(ab.data(), S, 2 * MAXM * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  TCI_TRY(tci_synchronize(ctx));
  const int k = (int)ctx->h_scalars[1];
  *ritz = ctx->h_scalars[2];
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
