// TCI "svd" and "trunc_svd" (App. C.2, Tensor linear algebra) on the device.
//
// The tensor is matricised (first k bonds = rows, I x J) and factored by the
// one-sided Jacobi method (Hestenes 1958; stable rotation formulas of
// Rutishauser, as in Demmel & Veselic, SIAM J. Matrix Anal. Appl. 13, 1992):
// the kappa = min(I, J) vectors along the longer dimension (columns of A'
// when J <= I, rows otherwise) are orthogonalised pairwise by plane rotations
// that are also applied to Q (initially the identity).  Each round of a sweep
// rotates kappa/2 disjoint pairs in parallel (round-robin order, one block of
// 128 threads per pair, row norms tracked so a pair needs one dot product;
// rows up to 1024 long are rotated from registers, longer ones in scaled
// form); sweeps repeat until no pair needs a rotation.  Small factorisations
// (vectors up to 64 long) run all their sweeps in one launch of a CTA cluster
// (a warp per pair, cluster barriers between rounds).  Then the norms of
// the vectors are the singular values, the normalised vectors one set of
// singular vectors and Q the other.  Arithmetic is FP64 for F64 and F32
// tensors.
//
// From kappa = 32 up, the Jacobi iteration is preconditioned as Drmac &
// Veselic (SIAM J. Matrix Anal. Appl. 29, 2008) do: a Householder QR with
// column pivoting of the m x n matrix whose columns are the n vectors,
// X P = H R, then one-sided Jacobi on the rows of R (R^T's columns).  On the
// graded matrices of truncation workloads the sweep count drops severalfold
// (about 30 to about 10 for an iTEBD two-site tensor).  With the converged
// rows sigma_i x_i^T = (Q' R)_i: X = sum_i (H [q'_i; 0]) sigma_i (P x_i)^T,
// so the length-m singular vectors are H applied to rows of Q' and the
// length-n ones are the permuted rows x_i.  For columns up to 256 long the
// whole QR runs in one cluster launch (a warp per column update).
//
// trunc_svd keeps chi values by the paper's rules: (a) drop s_i < s_min;
// (b) keep at least chi_min (or all that remain after (a)); (c) grow until the
// truncation error sum_{i >= chi} s_i^2 / sum_i s_i^2 <= target or
// chi = chi_max.  Singular vectors of zero singular values are returned as
// zero vectors.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "tci_internal.cuh"

namespace {

constexpr int kSvdT = 256;
constexpr int kMaxSweeps = 60;
constexpr int64_t kPrecondMin = 32;   // QR-precondition from this many vectors up
thread_local int t_last_sweeps = 0;   // Jacobi sweeps of the last factorisation (verbose report)

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One block of kRotT threads per pair (p, q): rows p and q of W (length m)
// and of Q (length nq).  The squared row norms are tracked in nrm2 (exact at
// the start of every sweep) and updated by Rutishauser's formulas
// ||x'||^2 = ||x||^2 - t g, ||y'||^2 = ||y||^2 + t g, so a pair costs one dot
// product instead of three: FP64 issue slots, not bytes, bound a round on
// B300.  A pair is rotated when |g| > tol ||x|| ||y|| (relative) and
// |g| > abs_tol (the rotation would move the matrix by more than rounding
// noise of its Frobenius norm); without the absolute test, vectors of
// negligible norm are re-rotated forever by the rounding noise of the large
// ones.  A sweep without rotations decides convergence on exact norms.
constexpr int kRotT = 128;

// Long rows (the generic round): plane rotations in scaled form.  A row is
// kept as d_i times its stored values (W and Q rows share d_i, which is 1 at
// the start of every sweep); rotating actual rows x = d_p x~, y = d_q y~ by
// (c, s = c t) gives x' = c d_p (x~ - t (d_q / d_p) y~) and
// y' = c d_q (y~ + t (d_p / d_q) x~), so the stored rows take one FMA per
// element each and the scales are multiplied by c (the fast Givens idea of
// Gentleman, 1973; the rounding error per element is the same as that of
// the explicit rotation).  A scale that would fall below 2^-400 is folded
// into its row by an explicit rotation instead.
__global__ void __launch_bounds__(kRotT) k_jacobi_round(double* __restrict__ W, int64_t m, double* __restrict__ Q,
                                                        int64_t nq, const int2* __restrict__ pairs,
                                                        double* __restrict__ nrm2, double* __restrict__ dsc,
                                                        double tol, double abs_tol, int* __restrict__ rotated) {
  const int2 pq = pairs[blockIdx.x];
  double* wp = W + (int64_t)pq.x * m;
  double* wq = W + (int64_t)pq.y * m;
  double g = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += kRotT) g = fma(wp[i], wq[i], g);
  __shared__ double red[kRotT / 32];
  __shared__ double cf[4];
  __shared__ int rot;
  g = warp_sum_d(g);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    double Gs = 0.0;
    for (int k = 0; k < kRotT / 32; ++k) Gs += red[k];
    const double dp = dsc[pq.x], dq = dsc[pq.y];
    const double G = dp * dq * Gs;
    const double A = nrm2[pq.x], B = nrm2[pq.y];
    rot = 0;
    if (fabs(G) > abs_tol && fabs(G) > tol * sqrt(A * B)) {
      const double zeta = (B - A) / (2.0 * G);
      const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      const double c = 1.0 / sqrt(1.0 + t * t);
      nrm2[pq.x] = fmax(A - t * G, 0.0);
      nrm2[pq.y] = B + t * G;
      const double np_ = c * dp, nq_ = c * dq;
      if (np_ > 0x1p-400 && nq_ > 0x1p-400) {
        cf[0] = -t * (dq / dp);   // x~' = x~ + cf0 y~
        cf[1] = t * (dp / dq);    // y~' = y~ + cf1 x~
        dsc[pq.x] = np_;
        dsc[pq.y] = nq_;
        rot = 1;
      } else {                    // explicit rotation of the actual rows, scales back to 1
        const double s = c * t;
        cf[0] = c * dp;
        cf[1] = -s * dq;
        cf[2] = s * dp;
        cf[3] = c * dq;
        dsc[pq.x] = 1.0;
        dsc[pq.y] = 1.0;
        rot = 2;
      }
      atomicExch(rotated, 1);
    }
  }
  __syncthreads();
  if (!rot) return;
  double* qp = Q + (int64_t)pq.x * nq;
  double* qq = Q + (int64_t)pq.y * nq;
  if (rot == 1) {
    const double f0 = cf[0], f1 = cf[1];
    for (int64_t i = threadIdx.x; i < m; i += kRotT) {
      const double x = wp[i], y = wq[i];
      wp[i] = fma(f0, y, x);
      wq[i] = fma(f1, x, y);
    }
    for (int64_t i = threadIdx.x; i < nq; i += kRotT) {
      const double x = qp[i], y = qq[i];
      qp[i] = fma(f0, y, x);
      qq[i] = fma(f1, x, y);
    }
  } else {
    const double a11 = cf[0], a12 = cf[1], a21 = cf[2], a22 = cf[3];
    for (int64_t i = threadIdx.x; i < m; i += kRotT) {
      const double x = wp[i], y = wq[i];
      wp[i] = fma(a11, x, a12 * y);
      wq[i] = fma(a21, x, a22 * y);
    }
    for (int64_t i = threadIdx.x; i < nq; i += kRotT) {
      const double x = qp[i], y = qq[i];
      qp[i] = fma(a11, x, a12 * y);
      qq[i] = fma(a21, x, a22 * y);
    }
  }
}

// Fold the scales into the rows (W and Q), reset them to 1 and take the exact
// squared norms of the W rows (one block per row).
__global__ void __launch_bounds__(kSvdT) k_fold_scales(double* __restrict__ W, int64_t m, double* __restrict__ Q,
                                                       int64_t nq, double* __restrict__ dsc,
                                                       double* __restrict__ sq) {
  const int64_t r = blockIdx.x;
  const double d = dsc[r];
  double* w = W + r * m;
  double* q = Q + r * nq;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += kSvdT) {
    const double x = d * w[i];
    if (d != 1.0) w[i] = x;
    a = fma(x, x, a);
  }
  if (d != 1.0)
    for (int64_t i = threadIdx.x; i < nq; i += kSvdT) q[i] *= d;
  __shared__ double red[kSvdT / 32];
  a = warp_sum_d(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kSvdT / 32; ++k) s += red[k];
    sq[r] = s;
    dsc[r] = 1.0;
  }
}

__global__ void k_fill(double* __restrict__ p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// The same round with both row pairs (W and Q) held in registers, E elements
// per thread (m, nq <= kRotT * E): every row is loaded once, before the
// reduction, and the squared norms are fetched at the same time, so a round
// costs one memory round trip instead of four.
template <int E>
__global__ void __launch_bounds__(kRotT) k_jacobi_round_reg(double* __restrict__ W, int64_t m,
                                                            double* __restrict__ Q, int64_t nq,
                                                            const int2* __restrict__ pairs,
                                                            double* __restrict__ nrm2, double tol, double abs_tol,
                                                            int* __restrict__ rotated) {
  const int2 pq = pairs[blockIdx.x];
  double* wp = W + (int64_t)pq.x * m;
  double* wq = W + (int64_t)pq.y * m;
  double* qp = Q + (int64_t)pq.x * nq;
  double* qq = Q + (int64_t)pq.y * nq;
  double A = 0.0, B = 0.0;
  if (threadIdx.x == 0) {
    A = nrm2[pq.x];
    B = nrm2[pq.y];
  }
  double x[E], y[E], u[E], v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t i = threadIdx.x + (int64_t)e * kRotT;
    x[e] = i < m ? wp[i] : 0.0;
    y[e] = i < m ? wq[i] : 0.0;
    u[e] = i < nq ? qp[i] : 0.0;
    v[e] = i < nq ? qq[i] : 0.0;
  }
  double g = 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) g = fma(x[e], y[e], g);
  __shared__ double red[kRotT / 32];
  __shared__ double cs[2];
  __shared__ int rot;
  g = warp_sum_d(g);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    double G = 0.0;
    for (int k = 0; k < kRotT / 32; ++k) G += red[k];
    rot = 0;
    if (fabs(G) > abs_tol && fabs(G) > tol * sqrt(A * B)) {
      const double zeta = (B - A) / (2.0 * G);
      const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      const double c = 1.0 / sqrt(1.0 + t * t);
      cs[0] = c;
      cs[1] = c * t;
      nrm2[pq.x] = fmax(A - t * G, 0.0);
      nrm2[pq.y] = B + t * G;
      rot = 1;
      atomicExch(rotated, 1);
    }
  }
  __syncthreads();
  if (!rot) return;
  const double c = cs[0], s = cs[1];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t i = threadIdx.x + (int64_t)e * kRotT;
    if (i < m) {
      wp[i] = c * x[e] - s * y[e];
      wq[i] = s * x[e] + c * y[e];
    }
    if (i < nq) {
      qp[i] = c * u[e] - s * v[e];
      qq[i] = s * u[e] + c * v[e];
    }
  }
}

// ---------------------------------------------------------------- small problems
// All sweeps of a small factorisation (rows and vectors at most 32 E long) in
// one launch of a cluster of CTAs: a warp per pair, the rounds separated by
// cluster barriers, exact norms at the start of every sweep, and the
// any-rotation test of a sweep combined across the cluster through
// distributed shared memory.  The rotation arithmetic is that of
// k_jacobi_round_reg.  Used where the rounds, not their FP64 work, set the
// time (one launch and one host read instead of a launch per round and a
// synchronisation per sweep).  info[0] = sweeps done, info[1] = converged.
namespace cg = cooperative_groups;
constexpr int kClT = 256;
constexpr int kClMax = 16;

template <int E>
__global__ void __launch_bounds__(kClT) k_jacobi_cluster(double* __restrict__ W, int64_t m, double* __restrict__ Q,
                                                        int64_t nq, int64_t n, const int2* __restrict__ pairs,
                                                        const int* __restrict__ start, int nrounds,
                                                        double* __restrict__ nrm2, double tol, double abs_tol,
                                                        int max_sweeps, int* __restrict__ info) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ int srot;
  const int lane = threadIdx.x & 31;
  const int nw = (int)cl.num_blocks() * (kClT / 32);
  const int gw = (int)cl.block_rank() * (kClT / 32) + (int)(threadIdx.x >> 5);
  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (threadIdx.x == 0) srot = 0;
    for (int64_t r = gw; r < n; r += nw) {   // exact squared norms
      const double* wr = W + r * m;
      double a = 0.0;
      for (int64_t i = lane; i < m; i += 32) a = fma(wr[i], wr[i], a);
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) nrm2[r] = a;
    }
    cl.sync();
    for (int rd = 0; rd < nrounds; ++rd) {
      const int p0 = start[rd], np = start[rd + 1] - p0;
      for (int k = gw; k < np; k += nw) {
        const int2 pq = pairs[p0 + k];
        double* wp = W + (int64_t)pq.x * m;
        double* wq = W + (int64_t)pq.y * m;
        double* qp = Q + (int64_t)pq.x * nq;
        double* qq = Q + (int64_t)pq.y * nq;
        const double A = nrm2[pq.x], B = nrm2[pq.y];   // issued with the row loads
        double x[E], y[E], u[E], v[E];
        double g = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int64_t i = lane + 32 * e;
          x[e] = i < m ? wp[i] : 0.0;
          y[e] = i < m ? wq[i] : 0.0;
          u[e] = i < nq ? qp[i] : 0.0;
          v[e] = i < nq ? qq[i] : 0.0;
          g = fma(x[e], y[e], g);
        }
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        __syncwarp();   // every lane has read the norms before lane 0 updates them
        if (fabs(g) > abs_tol && fabs(g) > tol * sqrt(A * B)) {   // the same decision in every lane
          const double zeta = (B - A) / (2.0 * g);
          const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          if (lane == 0) {
            nrm2[pq.x] = fmax(A - t * g, 0.0);
            nrm2[pq.y] = B + t * g;
            srot = 1;
          }
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int64_t i = lane + 32 * e;
            if (i < m) {
              wp[i] = c * x[e] - s * y[e];
              wq[i] = s * x[e] + c * y[e];
            }
            if (i < nq) {
              qp[i] = c * u[e] - s * v[e];
              qq[i] = s * u[e] + c * v[e];
            }
          }
        }
      }
      cl.sync();
    }
    // any rotation in this sweep, anywhere in the cluster (same answer in every CTA)
    int any = 0;
    for (int r = 0; r < (int)cl.num_blocks(); ++r) any |= *cl.map_shared_rank(&srot, r);
    converged = any == 0;
    cl.sync();   // every CTA has read every flag before the next sweep clears its own
  }
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    info[0] = sweep;
    info[1] = converged ? 1 : 0;
  }
}

// sq[r] = ||W_r||^2 (one block per row)
__global__ void __launch_bounds__(kSvdT) k_row_sumsq(const double* __restrict__ W, int64_t m, double* __restrict__ sq) {
  const double* w = W + (int64_t)blockIdx.x * m;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += kSvdT) a = fma(w[i], w[i], a);
  __shared__ double red[kSvdT / 32];
  a = warp_sum_d(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kSvdT / 32; ++k) s += red[k];
    sq[blockIdx.x] = s;
  }
}

// norms[r] = ||W_r|| (one block per row)
__global__ void __launch_bounds__(kSvdT) k_row_norms(const double* __restrict__ W, int64_t m, double* __restrict__ norms) {
  const double* w = W + (int64_t)blockIdx.x * m;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += kSvdT) a = fma(w[i], w[i], a);
  __shared__ double red[kSvdT / 32];
  a = warp_sum_d(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kSvdT / 32; ++k) s += red[k];
    norms[blockIdx.x] = sqrt(s);
  }
}

__global__ void k_identity(double* __restrict__ Q, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * n; i += (int64_t)gridDim.x * blockDim.x)
    Q[i] = (i / n == i % n) ? 1.0 : 0.0;
}

// dst[r * ncols + c] = src[perm[r] * ld + c] * scale(perm[r])   (selected rows, optionally normalised)
template <typename T>
__global__ void k_gather_rows(const double* __restrict__ src, int64_t ld, const int* __restrict__ perm, int rows,
                              int64_t ncols, const double* __restrict__ norms, int normalise, T* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * ncols;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ncols, c = i - r * ncols;
    const int pr = perm[r];
    double v = src[(int64_t)pr * ld + c];
    if (normalise) v = norms[pr] > 0.0 ? v / norms[pr] : 0.0;
    dst[i] = (T)v;
  }
}

// dst[c * rows + r] = src[perm[r] * ld + c] * scale   (selected rows, transposed)
template <typename T>
__global__ void k_gather_rows_t(const double* __restrict__ src, int64_t ld, const int* __restrict__ perm, int rows,
                                int64_t ncols, const double* __restrict__ norms, int normalise, T* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * ncols;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / rows, r = i - c * rows;
    const int pr = perm[r];
    double v = src[(int64_t)pr * ld + c];
    if (normalise) v = norms[pr] > 0.0 ? v / norms[pr] : 0.0;
    dst[i] = (T)v;
  }
}

// W[r * m + c] = A[c * lda_c + r * lda_r] converted to FP64
template <typename T>
__global__ void k_load_work(const T* __restrict__ A, int64_t rows, int64_t m, int64_t sr, int64_t sc,
                            double* __restrict__ W) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / m, c = i - r * m;
    W[i] = (double)A[r * sr + c * sc];
  }
}

// ---------------------------------------------------------------- QR with column pivoting
// The n vectors are the rows of W (length m); as a matrix X = W^T (m x n)
// they are its columns, stored contiguously.  Step k: pivot the remaining
// column of largest partial norm into position k, form the Householder
// reflector of X[k:, k] (LAPACK convention: v_k = 1, v stored below the
// diagonal, i.e. in W[k][k+1..], R[k][k] = beta in W[k][k], tau[k] = 0 when
// there is nothing below the diagonal) and apply it to the later columns.
constexpr int kQrT = 1024;

__device__ double block_sum_b(double v, double* red) {   // blockDim.x threads, result in every thread
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    red[32] = t;
  }
  __syncthreads();
  const double t = red[32];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kQrT) k_qr_pivot(double* __restrict__ W, int64_t m, int n, int k,
                                                   double* __restrict__ nrm2, int* __restrict__ qperm,
                                                   double* __restrict__ tau) {
  __shared__ double red[33];
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ int piv;
  // argmax of nrm2[k..n) (first index on ties)
  double best = -1.0;
  int besti = n;
  for (int j = k + threadIdx.x; j < n; j += kQrT) {
    const double x = nrm2[j];
    if (x > best) {
      best = x;
      besti = j;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, besti, o);
    if (ob > best || (ob == best && oi < besti)) {
      best = ob;
      besti = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    bv[threadIdx.x >> 5] = best;
    bi[threadIdx.x >> 5] = besti;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -1.0;
    int p = k;
    for (int i = 0; i < kQrT / 32; ++i)
      if (bi[i] < n && (bv[i] > b || (bv[i] == b && bi[i] < p))) {
        b = bv[i];
        p = bi[i];
      }
    piv = p;
  }
  __syncthreads();
  const int p = piv;
  if (p != k) {
    double* a = W + (int64_t)k * m;
    double* b = W + (int64_t)p * m;
    for (int64_t r = threadIdx.x; r < m; r += kQrT) {
      const double t = a[r];
      a[r] = b[r];
      b[r] = t;
    }
    if (threadIdx.x == 0) {
      const double t = nrm2[k];
      nrm2[k] = nrm2[p];
      nrm2[p] = t;
      const int q = qperm[k];
      qperm[k] = qperm[p];
      qperm[p] = q;
    }
    __syncthreads();
  }
  // Householder reflector of column k, rows k..m-1
  double* x = W + (int64_t)k * m;
  const double alpha = x[k];   // before the reduction's barriers: thread 0 overwrites x[k] below
  double sub = 0.0;
  for (int64_t r = k + 1 + threadIdx.x; r < m; r += kQrT) sub = fma(x[r], x[r], sub);
  sub = block_sum_b(sub, red);
  if (!(sub > 0.0)) {
    if (threadIdx.x == 0) tau[k] = 0.0;
    return;
  }
  const double beta = -copysign(sqrt(alpha * alpha + sub), alpha);
  const double scale = 1.0 / (alpha - beta);
  for (int64_t r = k + 1 + threadIdx.x; r < m; r += kQrT) x[r] *= scale;
  if (threadIdx.x == 0) {
    tau[k] = (beta - alpha) / beta;
    x[k] = beta;
  }
}

// One block per later column j = k + 1 + blockIdx.x: X[k:, j] -= tau v (v . X[k:, j]);
// then nrm2[j] = ||X[k+1:, j]||^2 (exact, so no norm downdating is needed).
__global__ void __launch_bounds__(kSvdT) k_qr_apply(double* __restrict__ W, int64_t m, int k,
                                                    double* __restrict__ nrm2, const double* __restrict__ tau) {
  __shared__ double red[33];
  const int j = k + 1 + blockIdx.x;
  const double* v = W + (int64_t)k * m;
  double* y = W + (int64_t)j * m;
  const double t = tau[k];
  if (t != 0.0) {
    double d = 0.0;
    for (int64_t r = k + 1 + threadIdx.x; r < m; r += kSvdT) d = fma(v[r], y[r], d);
    d = block_sum_b(d, red) + y[k];
    const double f = t * d;
    for (int64_t r = k + 1 + threadIdx.x; r < m; r += kSvdT) y[r] = fma(-f, v[r], y[r]);
    __syncthreads();
    if (threadIdx.x == 0) y[k] -= f;
  }
  double s2 = 0.0;
  for (int64_t r = k + 1 + threadIdx.x; r < m; r += kSvdT) s2 = fma(y[r], y[r], s2);
  s2 = block_sum_b(s2, red);
  if (threadIdx.x == 0) nrm2[j] = s2;
}

// The whole pivoted Householder QR (the k_qr_pivot / k_qr_apply steps for
// k = 0 .. n-1) in one launch of a cluster for columns up to 32 E long: per
// step, one warp picks the pivot, swaps and forms the reflector, a cluster
// barrier, then a warp per later column applies it and recomputes that
// column's norm, and another barrier.  Same arithmetic as the two kernels
// (warp instead of block sums).
template <int E>
__global__ void __launch_bounds__(kClT) k_qr_cluster(double* __restrict__ W, int64_t m, int n,
                                                    double* __restrict__ nrm2, int* __restrict__ qperm,
                                                    double* __restrict__ tau) {
  cg::cluster_group cl = cg::this_cluster();
  const int lane = threadIdx.x & 31;
  const int nw = (int)cl.num_blocks() * (kClT / 32);
  const int gw = (int)cl.block_rank() * (kClT / 32) + (int)(threadIdx.x >> 5);
  for (int k = 0; k < n; ++k) {
    if (gw == 0) {
      // argmax of nrm2[k..n) (first index on ties)
      double best = -1.0;
      int besti = n;
      for (int j = k + lane; j < n; j += 32) {
        const double x = nrm2[j];
        if (x > best) {
          best = x;
          besti = j;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
        if (ob > best || (ob == best && oi < besti)) {
          best = ob;
          besti = oi;
        }
      }
      const int p = besti < n ? besti : k;
      double* x = W + (int64_t)k * m;
      if (p != k) {
        double* b = W + (int64_t)p * m;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int64_t r = lane + 32 * e;
          if (r < m) {
            const double t = x[r];
            x[r] = b[r];
            b[r] = t;
          }
        }
        if (lane == 0) {
          const double t = nrm2[k];
          nrm2[k] = nrm2[p];
          nrm2[p] = t;
          const int q = qperm[k];
          qperm[k] = qperm[p];
          qperm[p] = q;
        }
        __syncwarp();
      }
      // Householder reflector of column k, rows k..m-1
      const double alpha = x[k];
      double sub = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t r = lane + 32 * e;
        if (r > k && r < m) sub = fma(x[r], x[r], sub);
      }
      for (int o = 16; o > 0; o >>= 1) sub += __shfl_xor_sync(0xffffffffu, sub, o);
      __syncwarp();   // every lane has read x[k] before lane 0 overwrites it
      if (!(sub > 0.0)) {
        if (lane == 0) tau[k] = 0.0;
      } else {
        const double beta = -copysign(sqrt(alpha * alpha + sub), alpha);
        const double scale = 1.0 / (alpha - beta);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int64_t r = lane + 32 * e;
          if (r > k && r < m) x[r] *= scale;
        }
        if (lane == 0) {
          tau[k] = (beta - alpha) / beta;
          x[k] = beta;
        }
      }
    }
    cl.sync();
    const double t = tau[k];
    const double* v = W + (int64_t)k * m;
    for (int j = k + 1 + gw; j < n; j += nw) {
      double* y = W + (int64_t)j * m;
      double vv[E], yy[E];
      double d = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t r = lane + 32 * e;
        const bool in = r > k && r < m;
        vv[e] = in ? v[r] : 0.0;
        yy[e] = in ? y[r] : 0.0;
        d = fma(vv[e], yy[e], d);
      }
      double s2 = 0.0;
      if (t != 0.0) {
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        const double yk = y[k];
        __syncwarp();   // every lane has read y[k] before lane 0 updates it
        const double f = t * (d + yk);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int64_t r = lane + 32 * e;
          if (r > k && r < m) {
            yy[e] = fma(-f, vv[e], yy[e]);
            y[r] = yy[e];
          }
        }
        if (lane == 0) y[k] = yk - f;
      }
#pragma unroll
      for (int e = 0; e < E; ++e) s2 = fma(yy[e], yy[e], s2);
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) nrm2[j] = s2;
    }
    cl.sync();
  }
}

// R (n x n, row-major, upper triangle): R[i][j] = X[i][j] = W[j][i] for i <= j.
__global__ void k_build_r(const double* __restrict__ W, int64_t m, int64_t n, double* __restrict__ R) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    R[e] = i <= j ? W[j * m + i] : 0.0;
  }
}

// Vn[i][qperm[c]] = Rj[i][c] / sigma_i: the length-n singular vectors, un-pivoted.
__global__ void k_unpivot_rows(const double* __restrict__ Rj, int64_t n, const double* __restrict__ sig,
                               const int* __restrict__ qperm, double* __restrict__ Vn) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, c = e - i * n;
    Vn[i * n + qperm[c]] = sig[i] > 0.0 ? Rj[e] / sig[i] : 0.0;
  }
}

// Uc[c] = [Q'[perm[c]]; 0] (chi rows of length m); zero for a zero singular value
__global__ void k_init_u(const double* __restrict__ Qj, int64_t n, const int* __restrict__ perm,
                         const double* __restrict__ sig, int64_t chi, int64_t m, double* __restrict__ Uc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < chi * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / m, r = e - c * m;
    const int pc = perm[c];
    Uc[e] = (r < n && sig[pc] > 0.0) ? Qj[(int64_t)pc * n + r] : 0.0;
  }
}

// One block per row c of Uc: Uc[c][k:] -= tau_k v_k (v_k . Uc[c][k:])  (H_k applied)
__global__ void __launch_bounds__(kSvdT) k_apply_h(const double* __restrict__ W, int64_t m, int k,
                                                   const double* __restrict__ tau, double* __restrict__ Uc) {
  __shared__ double red[33];
  const double t = tau[k];
  if (t == 0.0) return;
  const double* v = W + (int64_t)k * m;
  double* y = Uc + (int64_t)blockIdx.x * m;
  double d = 0.0;
  for (int64_t r = k + 1 + threadIdx.x; r < m; r += kSvdT) d = fma(v[r], y[r], d);
  d = block_sum_b(d, red) + y[k];
  const double f = t * d;
  for (int64_t r = k + 1 + threadIdx.x; r < m; r += kSvdT) y[r] = fma(-f, v[r], y[r]);
  __syncthreads();
  if (threadIdx.x == 0) y[k] -= f;
}

// All reflectors, last to first, for rows up to 32 E long: a warp per row c of
// Uc holds the row in registers and applies H_{n-1} .. H_0 in turn (rows are
// independent, so one launch replaces n); the arithmetic of k_apply_h.
template <int E>
__global__ void __launch_bounds__(kSvdT) k_apply_h_all(const double* __restrict__ W, int64_t m, int n,
                                                       const double* __restrict__ tau, double* __restrict__ Uc,
                                                       int64_t chi) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (kSvdT / 32) + (threadIdx.x >> 5);
  if (c >= chi) return;
  double* yrow = Uc + c * m;
  double y[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t r = lane + 32 * e;
    y[e] = r < m ? yrow[r] : 0.0;
  }
  for (int k = n - 1; k >= 0; --k) {
    const double t = tau[k];
    if (t == 0.0) continue;
    const double* v = W + (int64_t)k * m;
    double vv[E];
    double d = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t r = lane + 32 * e;
      vv[e] = (r > k && r < m) ? v[r] : 0.0;
      d = fma(vv[e], y[e], d);
    }
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    double yk = 0.0;   // y[k], held by lane k % 32 in element k / 32
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e == k / 32) yk = y[e];
    yk = __shfl_sync(0xffffffffu, yk, k & 31);
    const double f = t * (d + yk);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t r = lane + 32 * e;
      if (r > k && r < m) y[e] = fma(-f, vv[e], y[e]);
      else if (r == k) y[e] -= f;
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t r = lane + 32 * e;
    if (r < m) yrow[r] = y[e];
  }
}

__global__ void k_iota(int* __restrict__ p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int)i;
}

void launch_round(tci_context ctx, int np, double* W, int64_t m, double* Q, int64_t nq, const int2* pairs,
                  double* nrm2, double* dsc, double tol, double abs_tol, int* rotated) {
  const int64_t len = m > nq ? m : nq;
  if (len <= kRotT)
    k_jacobi_round_reg<1><<<np, kRotT, 0, ctx->stream>>>(W, m, Q, nq, pairs, nrm2, tol, abs_tol, rotated);
  else if (len <= 2 * kRotT)
    k_jacobi_round_reg<2><<<np, kRotT, 0, ctx->stream>>>(W, m, Q, nq, pairs, nrm2, tol, abs_tol, rotated);
  else if (len <= 4 * kRotT)
    k_jacobi_round_reg<4><<<np, kRotT, 0, ctx->stream>>>(W, m, Q, nq, pairs, nrm2, tol, abs_tol, rotated);
  else if (len <= 8 * kRotT)
    k_jacobi_round_reg<8><<<np, kRotT, 0, ctx->stream>>>(W, m, Q, nq, pairs, nrm2, tol, abs_tol, rotated);
  else   // longer rows: the register copies would cost occupancy (measured slower at 2048)
    k_jacobi_round<<<np, kRotT, 0, ctx->stream>>>(W, m, Q, nq, pairs, nrm2, dsc, tol, abs_tol, rotated);
}

bool round_uses_registers(int64_t m, int64_t nq) { return (m > nq ? m : nq) <= 8 * kRotT; }

// Cluster size for a kernel of kClT threads: 16 CTAs where the device allows
// non-portable clusters, else 8 (found once per kernel and device).
template <typename K>
int cluster_size_for(tci_context ctx, K* kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair((const void*)kernel, ctx->device);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int best = 8;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClMax;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kClMax);
    cfg.blockDim = dim3(kClT);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) == cudaSuccess && nclusters >= 1) best = kClMax;
  }
  cudaGetLastError();
  cache[key] = best;
  return best;
}

template <int E>
cudaError_t launch_jacobi_cluster_e(tci_context ctx, double* W, int64_t m, double* Q, int64_t n, const int2* pairs,
                                    const int* start, int nrounds, double* nrm2, double tol, double abs_tol,
                                    int max_sweeps, int* info) {
  const int ncl = cluster_size_for(ctx, k_jacobi_cluster<E>);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ncl);
  cfg.blockDim = dim3(kClT);
  cfg.stream = ctx->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_jacobi_cluster<E>, W, m, Q, n, n, pairs, start, nrounds, nrm2, tol, abs_tol,
                            max_sweeps, info);
}

template <int E>
cudaError_t launch_qr_cluster_e(tci_context ctx, double* W, int64_t m, int n, double* nrm2, int* qperm,
                                double* tau) {
  const int ncl = cluster_size_for(ctx, k_qr_cluster<E>);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ncl);
  cfg.blockDim = dim3(kClT);
  cfg.stream = ctx->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_qr_cluster<E>, W, m, n, nrm2, qperm, tau);
}

// The pivoted QR in one cluster launch for columns up to 256 long.
bool qr_clustered(int64_t m) { return m <= 8 * 32; }

cudaError_t launch_qr_cluster(tci_context ctx, double* W, int64_t m, int n, double* nrm2, int* qperm, double* tau) {
  if (m <= 32) return launch_qr_cluster_e<1>(ctx, W, m, n, nrm2, qperm, tau);
  if (m <= 64) return launch_qr_cluster_e<2>(ctx, W, m, n, nrm2, qperm, tau);
  if (m <= 128) return launch_qr_cluster_e<4>(ctx, W, m, n, nrm2, qperm, tau);
  return launch_qr_cluster_e<8>(ctx, W, m, n, nrm2, qperm, tau);
}

// All sweeps in one cluster launch when the rows and vectors are <= 64 long (measured:
// faster up to 32, even at 64, slower from 128, where a round has enough pairs to fill the GPU).
bool jacobi_clustered(int64_t m, int64_t n) { return (m > n ? m : n) <= 2 * 32 && n >= 2; }

cudaError_t launch_jacobi_cluster(tci_context ctx, double* W, int64_t m, double* Q, int64_t n, const int2* pairs,
                                  const int* start, int nrounds, double* nrm2, double tol, double abs_tol,
                                  int max_sweeps, int* info) {
  const int64_t len = m > n ? m : n;
  if (len <= 32)
    return launch_jacobi_cluster_e<1>(ctx, W, m, Q, n, pairs, start, nrounds, nrm2, tol, abs_tol, max_sweeps, info);
  if (len <= 64)
    return launch_jacobi_cluster_e<2>(ctx, W, m, Q, n, pairs, start, nrounds, nrm2, tol, abs_tol, max_sweeps, info);
  if (len <= 128)
    return launch_jacobi_cluster_e<4>(ctx, W, m, Q, n, pairs, start, nrounds, nrm2, tol, abs_tol, max_sweeps, info);
  return launch_jacobi_cluster_e<8>(ctx, W, m, Q, n, pairs, start, nrounds, nrm2, tol, abs_tol, max_sweeps, info);
}

int grid_of(tci_context ctx, int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)ctx->num_sms * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// Round-robin (circle method) schedule over n' = n rounded up to even
// indices: n'-1 rounds of n'/2 disjoint pairs; pairs touching the padding
// index n are left out.  Returns the pairs of all rounds and each round's start.
void round_robin(int n, std::vector<int2>& pairs, std::vector<int>& start) {
  const int np = n + (n & 1);
  std::vector<int> pos(np);
  std::iota(pos.begin(), pos.end(), 0);
  pairs.clear();
  start.assign(1, 0);
  for (int r = 0; r < np - 1; ++r) {
    for (int k = 0; k < np / 2; ++k) {
      int p = pos[k], q = pos[np - 1 - k];
      if (p >= n || q >= n) continue;
      if (p > q) std::swap(p, q);
      pairs.push_back(make_int2(p, q));
    }
    start.push_back((int)pairs.size());
    // keep pos[0], rotate the rest by one
    const int last = pos[np - 1];
    for (int k = np - 1; k > 1; --k) pos[k] = pos[k - 1];
    pos[1] = last;
  }
}

struct SvdWork {
  double* W = nullptr;
  double* Q = nullptr;
  double* norms = nullptr;
  int2* pairs = nullptr;
  int* flag = nullptr;
  int* info = nullptr;      // cluster sweeps: sweeps done, converged
  int* rstart = nullptr;    // cluster sweeps: first pair of each round
  int* perm = nullptr;
  // QR preconditioning
  double* R = nullptr;      // n x n: R, then the Jacobi vectors
  double* tau = nullptr;    // n Householder scalars
  double* nrm2 = nullptr;   // n partial column norms
  int* qperm = nullptr;     // n column pivots
  double* Vn = nullptr;     // n x n length-n singular vectors
  double* Uc = nullptr;     // chi x m length-m singular vectors (sorted)
  int* iota = nullptr;      // chi
  double* rn2 = nullptr;    // n tracked squared norms of the Jacobi rows
  double* dsc = nullptr;    // n row scales of the scaled rotations
  void free_all() {
    void* ps[] = {W, Q, norms, pairs, flag, info, rstart, perm, R, tau, nrm2, qperm, Vn, Uc, iota, rn2, dsc};
    for (void* p : ps) tci_dev_free(p);
  }
};

tci_status new_tensor_out(tci_context ctx, tci_dtype dt, int order, const int64_t* shape, tci_tensor* out) {
  if (*out && tci_ten_ok(*out)) tci_tensor_free(out);
  *out = nullptr;
  return tci_allocate(ctx, dt, order, shape, out);
}

// Factor a; chi_min < 0 means "no truncation" (plain svd).
tci_status svd_impl(tci_context ctx, tci_tensor a, int k, tci_tensor* u, tci_tensor* s, tci_tensor* vt, double* terr,
                    int64_t chi_min, int64_t chi_max, double target, double s_min) {
  if (!tci_ten_ok(a) || !u || !s || !vt) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "svd: invalid argument");
  if (a->dtype != TCI_F64 && a->dtype != TCI_F32)
    return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "svd: real tensors only in this build");
  if (k < 1 || k >= a->order) return tci_fail(ctx, TCI_ERR_SHAPE, "svd: need 1 <= num_of_bds_as_row < order");
  int64_t I = 1, J = 1;
  for (int i = 0; i < k; ++i) I *= a->shape[i];
  for (int i = k; i < a->order; ++i) J *= a->shape[i];
  const int64_t kappa = std::min(I, J);
  if (kappa > (1 << 20)) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "svd: matrix too large");
  tci_tensor src = a;
  tci_tensor tmp = nullptr;
  if (!tci_is_rowmajor(a)) {
    TCI_TRY(tci_copy(ctx, a, &tmp));
    src = tmp;
  }
  const bool cols = J <= I;             // orthogonalise the columns of A' (else its rows)
  const int64_t n = kappa, m = cols ? I : J;
  SvdWork w;
  auto fail = [&](tci_status st) {
    cudaStreamSynchronize(ctx->stream);
    w.free_all();
    if (tmp) tci_tensor_free(&tmp);
    return st;
  };
  tci_status st = TCI_OK;
  std::vector<int2> pairs;
  std::vector<int> start;
  round_robin((int)n, pairs, start);
  if ((st = tci_dev_alloc(ctx, sizeof(double) * n * m, (void**)&w.W)) != TCI_OK) return fail(st);
  if ((st = tci_dev_alloc(ctx, sizeof(double) * n * n, (void**)&w.Q)) != TCI_OK) return fail(st);
  if ((st = tci_dev_alloc(ctx, sizeof(double) * n, (void**)&w.norms)) != TCI_OK) return fail(st);
  if ((st = tci_dev_alloc(ctx, sizeof(int2) * std::max<size_t>(1, pairs.size()), (void**)&w.pairs)) != TCI_OK)
    return fail(st);
  if ((st = tci_dev_alloc(ctx, sizeof(int), (void**)&w.flag)) != TCI_OK) return fail(st);
  if ((st = tci_dev_alloc(ctx, sizeof(int) * n, (void**)&w.perm)) != TCI_OK) return fail(st);
  if (!pairs.empty()) {
    cudaError_t e = cudaMemcpyAsync(w.pairs, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: schedule"));
  }
  // W: the n vectors as rows (A'^T when orthogonalising columns)
  const int64_t sr = cols ? 1 : J, sc = cols ? J : 1;
  if (src->dtype == TCI_F64)
    k_load_work<double><<<grid_of(ctx, n * m), 256, 0, ctx->stream>>>((const double*)src->data, n, m, sr, sc, w.W);
  else
    k_load_work<float><<<grid_of(ctx, n * m), 256, 0, ctx->stream>>>((const float*)src->data, n, m, sr, sc, w.W);
  k_identity<<<grid_of(ctx, n * n), 256, 0, ctx->stream>>>(w.Q, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: setup"));
  // squared Frobenius norm for the absolute rotation threshold
  k_row_norms<<<(unsigned)n, kSvdT, 0, ctx->stream>>>(w.W, m, w.norms);
  std::vector<double> nrm0(n);
  e = cudaMemcpyAsync(nrm0.data(), w.norms, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: norms"));
  double fro2 = 0.0;
  for (double x : nrm0) fro2 += x * x;
  const double abs_tol = 1e-31 * fro2;   // ~ (machine epsilon * ||A||_F)^2
  // QR preconditioning (X P = H R); the Jacobi vectors become the rows of R
  const bool precond = n >= kPrecondMin;
  double* Wj = w.W;        // Jacobi vectors (n rows)
  int64_t mj = m;          // their length
  if (precond) {
    if ((st = tci_dev_alloc(ctx, sizeof(double) * n * n, (void**)&w.R)) != TCI_OK) return fail(st);
    if ((st = tci_dev_alloc(ctx, sizeof(double) * n, (void**)&w.tau)) != TCI_OK) return fail(st);
    if ((st = tci_dev_alloc(ctx, sizeof(double) * n, (void**)&w.nrm2)) != TCI_OK) return fail(st);
    if ((st = tci_dev_alloc(ctx, sizeof(int) * n, (void**)&w.qperm)) != TCI_OK) return fail(st);
    std::vector<double> n2(n);
    for (int64_t i = 0; i < n; ++i) n2[i] = nrm0[i] * nrm0[i];
    std::vector<int> qp(n);
    std::iota(qp.begin(), qp.end(), 0);
    e = cudaMemcpyAsync(w.nrm2, n2.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w.qperm, qp.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: QR set-up"));
    if (qr_clustered(m)) {
      e = launch_qr_cluster(ctx, w.W, m, (int)n, w.nrm2, w.qperm, w.tau);
      if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: QR"));
    } else {
      for (int64_t kk = 0; kk < n; ++kk) {
        k_qr_pivot<<<1, kQrT, 0, ctx->stream>>>(w.W, m, (int)n, (int)kk, w.nrm2, w.qperm, w.tau);
        if (kk + 1 < n)
          k_qr_apply<<<(unsigned)(n - kk - 1), kSvdT, 0, ctx->stream>>>(w.W, m, (int)kk, w.nrm2, w.tau);
      }
    }
    k_build_r<<<grid_of(ctx, n * n), 256, 0, ctx->stream>>>(w.W, m, n, w.R);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: QR"));
    Wj = w.R;
    mj = n;
  }
  const double tol = sqrt((double)mj) * 2.220446049250313e-16;
  int sweeps = 0;
  if (!w.rn2 && (st = tci_dev_alloc(ctx, sizeof(double) * n, (void**)&w.rn2)) != TCI_OK) return fail(st);
  const bool scaled = !round_uses_registers(mj, n);   // scaled rotations in the generic round
  if (scaled) {
    if ((st = tci_dev_alloc(ctx, sizeof(double) * n, (void**)&w.dsc)) != TCI_OK) return fail(st);
    k_fill<<<grid_of(ctx, n), 256, 0, ctx->stream>>>(w.dsc, n, 1.0);
  }
  if (!scaled && !pairs.empty() && jacobi_clustered(mj, n)) {
    const int nrounds = (int)start.size() - 1;
    if ((st = tci_dev_alloc(ctx, sizeof(int) * 2, (void**)&w.info)) != TCI_OK) return fail(st);
    if ((st = tci_dev_alloc(ctx, sizeof(int) * start.size(), (void**)&w.rstart)) != TCI_OK) return fail(st);
    e = cudaMemcpyAsync(w.rstart, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = launch_jacobi_cluster(ctx, Wj, mj, w.Q, n, w.pairs, w.rstart, nrounds, w.rn2, tol, abs_tol, kMaxSweeps,
                                w.info);
    int info[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(info, w.info, sizeof(info), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: cluster sweeps"));
    sweeps = info[1] ? info[0] - 1 : kMaxSweeps;   // as the loop below counts: sweeps that rotated
    pairs.clear();   // done: skip the per-round loop below
  }
  for (; sweeps < kMaxSweeps && !pairs.empty(); ++sweeps) {
    cudaMemsetAsync(w.flag, 0, sizeof(int), ctx->stream);
    // exact norms each sweep (scales folded into the rows first)
    if (scaled)
      k_fold_scales<<<(unsigned)n, kSvdT, 0, ctx->stream>>>(Wj, mj, w.Q, n, w.dsc, w.rn2);
    else
      k_row_sumsq<<<(unsigned)n, kSvdT, 0, ctx->stream>>>(Wj, mj, w.rn2);
    for (size_t r = 0; r + 1 < start.size(); ++r) {
      const int np = start[r + 1] - start[r];
      if (np > 0)
        launch_round(ctx, np, Wj, mj, w.Q, n, w.pairs + start[r], w.rn2, w.dsc, tol, abs_tol, w.flag);
    }
    int rotated = 0;
    e = cudaMemcpyAsync(&rotated, w.flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: sweep"));
    if (!rotated) break;
  }
  if (sweeps == kMaxSweeps) return fail(tci_fail(ctx, TCI_ERR_TIMEOUT, "svd: Jacobi sweeps did not converge"));
  if (scaled) k_fold_scales<<<(unsigned)n, kSvdT, 0, ctx->stream>>>(Wj, mj, w.Q, n, w.dsc, w.rn2);
  t_last_sweeps = sweeps;
  // singular values, sorted
  k_row_norms<<<(unsigned)n, kSvdT, 0, ctx->stream>>>(Wj, mj, w.norms);
  std::vector<double> sv(n);
  e = cudaMemcpyAsync(sv.data(), w.norms, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: norms"));
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return sv[x] > sv[y]; });
  std::vector<double> sorted(n);
  for (int64_t i = 0; i < n; ++i) sorted[i] = sv[perm[i]];
  // retained count (paper's rules a-c) and truncation error
  int64_t chi = n;
  double tot = 0.0;
  for (double x : sorted) tot += x * x;
  if (chi_min >= 0) {
    int64_t remain = 0;
    for (double x : sorted) remain += x >= s_min ? 1 : 0;
    const int64_t cmin = std::min(chi_min, chi_max);
    if (remain <= cmin) {
      chi = remain;
    } else {
      chi = cmin;
      std::vector<double> tail(n + 1, 0.0);   // tail[c] = sum_{i >= c} s_i^2
      for (int64_t i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + sorted[i] * sorted[i];
      auto err_of = [&](int64_t c) { return tot > 0.0 ? tail[c] / tot : 0.0; };
      while (chi < std::min(chi_max, remain) && err_of(chi) > target) ++chi;
    }
  }
  if (terr) {
    double t = 0.0;
    for (int64_t i = chi; i < n; ++i) t += sorted[i] * sorted[i];
    *terr = tot > 0.0 ? t / tot : 0.0;
  }
  e = cudaMemcpyAsync(w.perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: permutation"));
  // outputs
  const tci_dtype dt = a->dtype;
  int64_t ushape[TCI_MAX_ORDER], vshape[TCI_MAX_ORDER];
  for (int i = 0; i < k; ++i) ushape[i] = a->shape[i];
  ushape[k] = chi;
  vshape[0] = chi;
  for (int i = k; i < a->order; ++i) vshape[1 + i - k] = a->shape[i];
  if ((st = new_tensor_out(ctx, dt, k + 1, ushape, u)) != TCI_OK) return fail(st);
  if ((st = new_tensor_out(ctx, dt, 1, &chi, s)) != TCI_OK) return fail(st);
  if ((st = new_tensor_out(ctx, dt, a->order - k + 1, vshape, vt)) != TCI_OK) return fail(st);
  if (chi > 0) {
    // sorted singular values
    if (dt == TCI_F64) {
      e = cudaMemcpyAsync((*s)->data, sorted.data(), sizeof(double) * chi, cudaMemcpyHostToDevice, ctx->stream);
    } else {
      std::vector<float> sf(sorted.begin(), sorted.begin() + chi);
      e = cudaMemcpyAsync((*s)->data, sf.data(), sizeof(float) * chi, cudaMemcpyHostToDevice, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: values"));
    const int g1 = grid_of(ctx, chi * m), g2 = grid_of(ctx, chi * n);
    // Length-m singular vectors LM (unit after normalising by norms when normLM) and
    // length-n ones LN, each addressed through a row permutation.
    const double* LM = Wj;
    const int* permLM = w.perm;
    int normLM = 1;
    const double* LN = w.Q;
    if (precond) {
      // length-n: the converged rows of R, normalised and un-pivoted
      if ((st = tci_dev_alloc(ctx, sizeof(double) * n * n, (void**)&w.Vn)) != TCI_OK) return fail(st);
      k_unpivot_rows<<<grid_of(ctx, n * n), 256, 0, ctx->stream>>>(Wj, n, w.norms, w.qperm, w.Vn);
      // length-m: H [q'_c; 0] for the kept c, reflectors applied last to first
      if ((st = tci_dev_alloc(ctx, sizeof(double) * chi * m, (void**)&w.Uc)) != TCI_OK) return fail(st);
      if ((st = tci_dev_alloc(ctx, sizeof(int) * chi, (void**)&w.iota)) != TCI_OK) return fail(st);
      k_init_u<<<grid_of(ctx, chi * m), 256, 0, ctx->stream>>>(w.Q, n, w.perm, w.norms, chi, m, w.Uc);
      k_iota<<<grid_of(ctx, chi), 256, 0, ctx->stream>>>(w.iota, chi);
      const unsigned hb = (unsigned)((chi + kSvdT / 32 - 1) / (kSvdT / 32));
      if (m <= 32)
        k_apply_h_all<1><<<hb, kSvdT, 0, ctx->stream>>>(w.W, m, (int)n, w.tau, w.Uc, chi);
      else if (m <= 64)
        k_apply_h_all<2><<<hb, kSvdT, 0, ctx->stream>>>(w.W, m, (int)n, w.tau, w.Uc, chi);
      else if (m <= 128)
        k_apply_h_all<4><<<hb, kSvdT, 0, ctx->stream>>>(w.W, m, (int)n, w.tau, w.Uc, chi);
      else if (m <= 256)
        k_apply_h_all<8><<<hb, kSvdT, 0, ctx->stream>>>(w.W, m, (int)n, w.tau, w.Uc, chi);
      else
        for (int64_t kk = n - 1; kk >= 0; --kk)
          k_apply_h<<<(unsigned)chi, kSvdT, 0, ctx->stream>>>(w.W, m, (int)kk, w.tau, w.Uc);
      LM = w.Uc;
      permLM = w.iota;
      normLM = 0;
      LN = w.Vn;
    }
    // cols: U[i][c] = LM[c][i] (transposed gather), V^T rows = LN rows.
    // rows: U[i][c] = LN[c][i] (transposed gather), V^T rows = LM rows.
    if (dt == TCI_F64) {
      double* U = (double*)(*u)->data;
      double* Vt = (double*)(*vt)->data;
      if (cols) {
        k_gather_rows_t<double><<<g1, 256, 0, ctx->stream>>>(LM, m, permLM, (int)chi, m, w.norms, normLM, U);
        k_gather_rows<double><<<g2, 256, 0, ctx->stream>>>(LN, n, w.perm, (int)chi, n, w.norms, 0, Vt);
      } else {
        k_gather_rows_t<double><<<g2, 256, 0, ctx->stream>>>(LN, n, w.perm, (int)chi, n, w.norms, 0, U);
        k_gather_rows<double><<<g1, 256, 0, ctx->stream>>>(LM, m, permLM, (int)chi, m, w.norms, normLM, Vt);
      }
    } else {
      float* U = (float*)(*u)->data;
      float* Vt = (float*)(*vt)->data;
      if (cols) {
        k_gather_rows_t<float><<<g1, 256, 0, ctx->stream>>>(LM, m, permLM, (int)chi, m, w.norms, normLM, U);
        k_gather_rows<float><<<g2, 256, 0, ctx->stream>>>(LN, n, w.perm, (int)chi, n, w.norms, 0, Vt);
      } else {
        k_gather_rows_t<float><<<g2, 256, 0, ctx->stream>>>(LN, n, w.perm, (int)chi, n, w.norms, 0, U);
        k_gather_rows<float><<<g1, 256, 0, ctx->stream>>>(LM, m, permLM, (int)chi, m, w.norms, normLM, Vt);
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: outputs"));
  }
  return fail(TCI_OK);
}

}  // namespace

extern "C" tci_status tci_svd(tci_context ctx, tci_tensor a, int num_of_bds_as_row, tci_tensor* u, tci_tensor* s,
                              tci_tensor* v_dag) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "svd");
  if (tci_ten_ok(a)) vs.info = tci_shape_str(a);
  t_last_sweeps = 0;
  const tci_status st = svd_impl(ctx, a, num_of_bds_as_row, u, s, v_dag, nullptr, -1, 0, 0.0, 0.0);
  vs.info += " sweeps=" + std::to_string(t_last_sweeps);
  return st;
}

extern "C" tci_status tci_trunc_svd(tci_context ctx, tci_tensor a, int num_of_bds_as_row, tci_tensor* u,
                                    tci_tensor* s, tci_tensor* v_dag, double* trunc_err, int64_t chi_min,
                                    int64_t chi_max, double target_trunc_err, double s_min) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "trunc_svd");
  if (tci_ten_ok(a)) vs.info = tci_shape_str(a);
  if (chi_min < 1 || chi_max < 1) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "trunc_svd: chi_min and chi_max must be >= 1");
  t_last_sweeps = 0;
  const tci_status st =
      svd_impl(ctx, a, num_of_bds_as_row, u, s, v_dag, trunc_err, chi_min, chi_max, target_trunc_err, s_min);
  vs.info += " sweeps=" + std::to_string(t_last_sweeps);
  return st;
}
