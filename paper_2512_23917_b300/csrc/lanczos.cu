// Lanczos ground-state solve of H_eff with FP64 vector arithmetic on the
// device (textbook: Golub & Van Loan Sec. 10.1; classical Gram-Schmidt
// applied twice for full re-orthogonalisation; Sturm-sequence bisection,
// Sec. 8.4, and inverse iteration for the tridiagonal eigenpair).
//
// All scalars (alpha, beta, re-orthogonalisation coefficients, stop flag,
// step count, Ritz coefficients) stay in device memory; the host enqueues
// the whole sequence and reads back once at the end.  Reductions are
// deterministic: a fixed grid, a fixed per-thread order and an in-order sum
// of the block partials.
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
constexpr int NSCAL = 4 * MAXM + 32;

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
  double* V = p->lz_V;
  double* w = p->lz_w;
  double* part = p->lz_part;
  const double tol = 1e-12;

  k_init_scal<<<1, 256, 0, ctx->stream>>>(S);
  // v0 = psi0 / ||psi0||
  k_sumsq<<<NB, NT, 0, ctx->stream>>>((const double*)psi0->data, n, part, ctrl);
  k_reduce_parts<<<1, 256, 0, ctx->stream>>>(part, 1, ctrl + 3, ctrl);
  k_start_vec<<<NB, NT, 0, ctx->stream>>>((const double*)psi0->data, V, n, S);
  TCI_CUDA(ctx, cudaGetLastError());
  for (int j = 0; j < nsteps; ++j) {
    double* vj = V + (int64_t)j * ldv;
    TCI_TRY(tci_heff_apply_raw(p, vj, w, false));
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
  if (x) k_ritz_vec<<<NB, NT, 0, ctx->stream>>>(V, ldv, S, (double*)x->data, n);
  TCI_CUDA(ctx, cudaGetLastError());
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
