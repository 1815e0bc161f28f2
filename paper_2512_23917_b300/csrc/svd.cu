// TCI "svd" and "trunc_svd" (App. C.2, Tensor linear algebra) on the device.
//
// The tensor is matricised (first k bonds = rows, I x J) and factored by the
// one-sided Jacobi method (Hestenes 1958; stable rotation formulas of
// Rutishauser, as in Demmel & Veselic, SIAM J. Matrix Anal. Appl. 13, 1992):
// the kappa = min(I, J) vectors along the longer dimension (columns of A'
// when J <= I, rows otherwise) are orthogonalised pairwise by plane rotations
// that are also applied to Q (initially the identity).  Each round of a sweep
// rotates kappa/2 disjoint pairs in parallel (round-robin order, one block per
// pair); sweeps repeat until no pair needs a rotation.  Then the norms of the
// vectors are the singular values, the normalised vectors one set of singular
// vectors and Q the other.  Arithmetic is FP64 for F64 and F32 tensors.
//
// trunc_svd keeps chi values by the paper's rules: (a) drop s_i < s_min;
// (b) keep at least chi_min (or all that remain after (a)); (c) grow until the
// truncation error sum_{i >= chi} s_i^2 / sum_i s_i^2 <= target or
// chi = chi_max.  Singular vectors of zero singular values are returned as
// zero vectors.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "tci_internal.cuh"

namespace {

constexpr int kSvdT = 256;
constexpr int kMaxSweeps = 60;

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One block per pair (p, q): rows p and q of W (length m) and of Q (length nq).
// A pair is rotated when |g| > tol ||x|| ||y|| (relative) and |g| > abs_tol
// (the rotation would move the matrix by more than rounding noise of its
// Frobenius norm); without the absolute test, vectors of negligible norm are
// re-rotated forever by the rounding noise of the large ones.
__global__ void __launch_bounds__(kSvdT) k_jacobi_round(double* __restrict__ W, int64_t m, double* __restrict__ Q,
                                                        int64_t nq, const int2* __restrict__ pairs, double tol,
                                                        double abs_tol, int* __restrict__ rotated) {
  const int2 pq = pairs[blockIdx.x];
  double* wp = W + (int64_t)pq.x * m;
  double* wq = W + (int64_t)pq.y * m;
  double a = 0.0, b = 0.0, g = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += kSvdT) {
    const double x = wp[i], y = wq[i];
    a = fma(x, x, a);
    b = fma(y, y, b);
    g = fma(x, y, g);
  }
  __shared__ double red[3][kSvdT / 32];
  __shared__ double cs[2];
  __shared__ int rot;
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  g = warp_sum_d(g);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
    red[2][wid] = g;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, B = 0.0, G = 0.0;
    for (int k = 0; k < kSvdT / 32; ++k) {
      A += red[0][k];
      B += red[1][k];
      G += red[2][k];
    }
    rot = 0;
    if (fabs(G) > abs_tol && fabs(G) > tol * sqrt(A * B)) {
      const double zeta = (B - A) / (2.0 * G);
      const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      const double c = 1.0 / sqrt(1.0 + t * t);
      cs[0] = c;
      cs[1] = c * t;
      rot = 1;
      atomicExch(rotated, 1);
    }
  }
  __syncthreads();
  if (!rot) return;
  const double c = cs[0], s = cs[1];
  for (int64_t i = threadIdx.x; i < m; i += kSvdT) {
    const double x = wp[i], y = wq[i];
    wp[i] = c * x - s * y;
    wq[i] = s * x + c * y;
  }
  double* qp = Q + (int64_t)pq.x * nq;
  double* qq = Q + (int64_t)pq.y * nq;
  for (int64_t i = threadIdx.x; i < nq; i += kSvdT) {
    const double x = qp[i], y = qq[i];
    qp[i] = c * x - s * y;
    qq[i] = s * x + c * y;
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
  int* perm = nullptr;
  void free_all() {
    void* ps[] = {W, Q, norms, pairs, flag, perm};
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
  const double tol = sqrt((double)m) * 2.220446049250313e-16;
  // squared Frobenius norm for the absolute rotation threshold
  k_row_norms<<<(unsigned)n, kSvdT, 0, ctx->stream>>>(w.W, m, w.norms);
  std::vector<double> nrm0(n);
  e = cudaMemcpyAsync(nrm0.data(), w.norms, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: norms"));
  double fro2 = 0.0;
  for (double x : nrm0) fro2 += x * x;
  const double abs_tol = 1e-31 * fro2;   // ~ (machine epsilon * ||A||_F)^2
  int sweeps = 0;
  for (; sweeps < kMaxSweeps && !pairs.empty(); ++sweeps) {
    cudaMemsetAsync(w.flag, 0, sizeof(int), ctx->stream);
    for (size_t r = 0; r + 1 < start.size(); ++r) {
      const int np = start[r + 1] - start[r];
      if (np > 0)
        k_jacobi_round<<<np, kSvdT, 0, ctx->stream>>>(w.W, m, w.Q, n, w.pairs + start[r], tol, abs_tol, w.flag);
    }
    int rotated = 0;
    e = cudaMemcpyAsync(&rotated, w.flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(tci_cuda_fail(ctx, e, "svd: sweep"));
    if (!rotated) break;
  }
  if (sweeps == kMaxSweeps) return fail(tci_fail(ctx, TCI_ERR_TIMEOUT, "svd: Jacobi sweeps did not converge"));
  // singular values, sorted
  k_row_norms<<<(unsigned)n, kSvdT, 0, ctx->stream>>>(w.W, m, w.norms);
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
    // cols: U[i][c] = W[perm c][i] / s (transposed gather), V^T rows = Q rows.
    // rows: U[i][c] = Q[perm c][i] (transposed gather), V^T rows = W rows / s.
    if (dt == TCI_F64) {
      double* U = (double*)(*u)->data;
      double* Vt = (double*)(*vt)->data;
      if (cols) {
        k_gather_rows_t<double><<<g1, 256, 0, ctx->stream>>>(w.W, m, w.perm, (int)chi, m, w.norms, 1, U);
        k_gather_rows<double><<<g2, 256, 0, ctx->stream>>>(w.Q, n, w.perm, (int)chi, n, w.norms, 0, Vt);
      } else {
        k_gather_rows_t<double><<<g2, 256, 0, ctx->stream>>>(w.Q, n, w.perm, (int)chi, n, w.norms, 0, U);
        k_gather_rows<double><<<g1, 256, 0, ctx->stream>>>(w.W, m, w.perm, (int)chi, m, w.norms, 1, Vt);
      }
    } else {
      float* U = (float*)(*u)->data;
      float* Vt = (float*)(*vt)->data;
      if (cols) {
        k_gather_rows_t<float><<<g1, 256, 0, ctx->stream>>>(w.W, m, w.perm, (int)chi, m, w.norms, 1, U);
        k_gather_rows<float><<<g2, 256, 0, ctx->stream>>>(w.Q, n, w.perm, (int)chi, n, w.norms, 0, Vt);
      } else {
        k_gather_rows_t<float><<<g2, 256, 0, ctx->stream>>>(w.Q, n, w.perm, (int)chi, n, w.norms, 0, U);
        k_gather_rows<float><<<g1, 256, 0, ctx->stream>>>(w.W, m, w.perm, (int)chi, m, w.norms, 1, Vt);
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
  return svd_impl(ctx, a, num_of_bds_as_row, u, s, v_dag, nullptr, -1, 0, 0.0, 0.0);
}

extern "C" tci_status tci_trunc_svd(tci_context ctx, tci_tensor a, int num_of_bds_as_row, tci_tensor* u,
                                    tci_tensor* s, tci_tensor* v_dag, double* trunc_err, int64_t chi_min,
                                    int64_t chi_max, double target_trunc_err, double s_min) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "trunc_svd");
  if (tci_ten_ok(a)) vs.info = tci_shape_str(a);
  if (chi_min < 1 || chi_max < 1) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "trunc_svd: chi_min and chi_max must be >= 1");
  return svd_impl(ctx, a, num_of_bds_as_row, u, s, v_dag, trunc_err, chi_min, chi_max, target_trunc_err, s_min);
}
