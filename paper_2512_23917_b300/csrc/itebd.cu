// iTEBD ground-state iteration of the paper's App. A on the device, driven
// from the host through the library's own calls (diag, contract, norm,
// trunc_svd, normalize).  Iteration i uses A = i mod 2, B = (i + 1) mod 2:
//
//   Theta  = diag(L_B) Gamma_A diag(L_A) Gamma_B diag(L_B)      [chi, d, d, chi]
//   Theta' = Theta contracted with the gate u = exp(-dt h) over Theta's two
//            physical bonds and u's first two bonds
//   Gamma_A, L_A, Gamma_B = trunc_svd(Theta', 2, chi_min 1, chi, 0, s_min)
//   L_A /= ||L_A||;  Gamma_A = diag(1/L_B) Gamma_A;  Gamma_B = Gamma_B diag(1/L_B)
//   E_i = -log ||Theta'||^2 / (2 dt)   (energy per bond = per site)
//
// The gate is formed on the device from h by scaling and squaring with a
// truncated Taylor series (Moler & Van Loan, SIAM Rev. 45, 2003, method 3).
#include <math.h>

#include "tci_internal.cuh"

namespace {


// u = exp(-dt h) for a 4 x 4 h (one thread): scale by 2^-s so ||A||_1 <= 1/2,
// Taylor series to degree 18, then square s times.
__global__ void k_expm4(const double* __restrict__ h, double dt, double* __restrict__ u) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double A[16], T[16], P[16], Q[16];
  double norm1 = 0.0;
  for (int j = 0; j < 4; ++j) {
    double c = 0.0;
    for (int i = 0; i < 4; ++i) c += fabs(h[i * 4 + j]);
    norm1 = fmax(norm1, c);
  }
  norm1 *= fabs(dt);
  int s = 0;
  while (norm1 > 0.5 && s < 60) {
    norm1 *= 0.5;
    ++s;
  }
  const double scale = -dt * ldexp(1.0, -s);
  for (int i = 0; i < 16; ++i) {
    A[i] = scale * h[i];
    T[i] = (i % 5 == 0) ? 1.0 : 0.0;   // identity
    P[i] = T[i];
  }
  for (int k = 1; k <= 18; ++k) {   // P = P A / k; T += P
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        double acc = 0.0;
        for (int l = 0; l < 4; ++l) acc += P[i * 4 + l] * A[l * 4 + j];
        Q[i * 4 + j] = acc / k;
      }
    for (int i = 0; i < 16; ++i) {
      P[i] = Q[i];
      T[i] += P[i];
    }
  }
  for (int r = 0; r < s; ++r) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        double acc = 0.0;
        for (int l = 0; l < 4; ++l) acc += T[i * 4 + l] * T[l * 4 + j];
        Q[i * 4 + j] = acc;
      }
    for (int i = 0; i < 16; ++i) T[i] = Q[i];
  }
  for (int i = 0; i < 16; ++i) u[i] = T[i];
}

__global__ void k_reciprocal(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = 1.0 / x[i];
}

tci_status contract_new(tci_context ctx, tci_tensor a, const char* la, tci_tensor b, const char* lb, const char* lc,
                        tci_tensor* out) {
  *out = nullptr;
  return tci_contract(ctx, a, la, b, lb, out, lc);
}

// Replace dst's metadata and storage by src's (src is consumed).
void take_storage(tci_context ctx, tci_tensor dst, tci_tensor src) {
  (void)ctx;
  tci_dev_free(dst->alloc);   // stream-ordered: after the work already queued on it
  dst->dtype = src->dtype;
  dst->order = src->order;
  for (int i = 0; i < src->order; ++i) {
    dst->shape[i] = src->shape[i];
    dst->strides[i] = src->strides[i];
  }
  dst->data = src->data;
  dst->alloc = src->alloc;
  dst->device = src->device;
  src->alloc = nullptr;
  tci_tensor_free(&src);
}

bool f64_rowmajor(tci_tensor t) { return tci_ten_ok(t) && t->dtype == TCI_F64 && tci_is_rowmajor(t); }

}  // namespace

extern "C" tci_status tci_itebd(tci_context ctx, tci_tensor h, double dt, tci_tensor gamma_a, tci_tensor gamma_b,
                                tci_tensor lambda_a, tci_tensor lambda_b, int64_t chi, double s_min, int niters,
                                double* energies, double* trunc_errs) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "itebd");
  if (!f64_rowmajor(h) || tci_numel(h) != 16)
    return tci_fail(ctx, TCI_ERR_SHAPE, "itebd: h must be a row-major F64 [4, 4] (or [2, 2, 2, 2]) tensor");
  tci_tensor G[2] = {gamma_a, gamma_b}, Lm[2] = {lambda_a, lambda_b};
  for (int q = 0; q < 2; ++q) {
    if (!f64_rowmajor(G[q]) || G[q]->order != 3 || G[q]->shape[1] != 2)
      return tci_fail(ctx, TCI_ERR_SHAPE, "itebd: Gamma tensors must be row-major F64 [chi, 2, chi]");
    if (!f64_rowmajor(Lm[q]) || Lm[q]->order != 1)
      return tci_fail(ctx, TCI_ERR_SHAPE, "itebd: Lambda tensors must be F64 vectors");
  }
  if (G[0]->shape[0] != Lm[1]->shape[0] || G[0]->shape[2] != Lm[0]->shape[0] || G[1]->shape[0] != Lm[0]->shape[0] ||
      G[1]->shape[2] != Lm[1]->shape[0])
    return tci_fail(ctx, TCI_ERR_SHAPE, "itebd: unit-cell bond dimensions do not match");
  if (chi < 1 || niters < 0 || !(dt > 0.0) || (niters > 0 && !energies))
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "itebd: need chi >= 1, dt > 0, niters >= 0 and an energy buffer");
  vs.info = "chi=" + std::to_string(chi) + " iters=" + std::to_string(niters);
  TciOwned u;
  const int64_t ushape[4] = {2, 2, 2, 2};
  TCI_TRY(tci_allocate(ctx, TCI_F64, 4, ushape, &u.t));
  k_expm4<<<1, 32, 0, ctx->stream>>>((const double*)h->data, dt, (double*)u.t->data);
  TCI_CUDA(ctx, cudaGetLastError());
  for (int i = 0; i < niters; ++i) {
    const int A = i % 2, B = (i + 1) % 2;
    TciOwned la, lb, t1, t2, t3, t4, th, ua, sa, vb, linv, linvd;
    TCI_TRY(tci_diag_to(ctx, Lm[A], &la.t));
    TCI_TRY(tci_diag_to(ctx, Lm[B], &lb.t));
    TCI_TRY(contract_new(ctx, lb.t, "ij", G[A], "jkl", "ikl", &t1.t));
    TCI_TRY(contract_new(ctx, t1.t, "ijk", la.t, "kl", "ijl", &t2.t));
    TCI_TRY(contract_new(ctx, t2.t, "ijk", G[B], "klm", "ijlm", &t3.t));
    TCI_TRY(contract_new(ctx, t3.t, "ijkl", lb.t, "lm", "ijkm", &t4.t));
    TCI_TRY(contract_new(ctx, t4.t, "ijkl", u.t, "jkmn", "imnl", &th.t));
    double nrm = 0.0;
    TCI_TRY(tci_norm(ctx, th.t, &nrm));
    energies[i] = -log(nrm * nrm) / dt / 2.0;
    double terr = 0.0;
    TCI_TRY(tci_trunc_svd(ctx, th.t, 2, &ua.t, &sa.t, &vb.t, &terr, 1, chi, 0.0, s_min));
    if (trunc_errs) trunc_errs[i] = terr;
    TCI_TRY(tci_normalize(ctx, sa.t, nullptr));
    const int64_t nb = Lm[B]->shape[0];
    TCI_TRY(tci_allocate(ctx, TCI_F64, 1, &nb, &linv.t));
    k_reciprocal<<<(unsigned)((nb + 255) / 256), 256, 0, ctx->stream>>>((const double*)Lm[B]->data,
                                                                      (double*)linv.t->data, nb);
    TCI_CUDA(ctx, cudaGetLastError());
    TCI_TRY(tci_diag_to(ctx, linv.t, &linvd.t));
    tci_tensor ga = nullptr, gb = nullptr;
    TCI_TRY(contract_new(ctx, linvd.t, "ij", ua.t, "jkl", "ikl", &ga));
    take_storage(ctx, G[A], ga);
    TCI_TRY(contract_new(ctx, vb.t, "ijk", linvd.t, "kl", "ijl", &gb));
    take_storage(ctx, G[B], gb);
    take_storage(ctx, Lm[A], sa.t);
    sa.t = nullptr;
  }
  return tci_synchronize(ctx);
}
