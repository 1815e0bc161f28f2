// Two-site finite DMRG for an open chain with a uniform MPO, driven from the
// host through the library's own calls: TCI contract (environment updates and
// two-site tensors), the H_eff plan and its Lanczos solver, TCI trunc_svd.
// The paper names DMRG as a target of TCI (Sec. I); the sweep is the textbook
// one (Schollwoeck, Ann. Phys. 326, 96 (2011), Secs. 6.2-6.4):
//
//   start: Neel product state A_k[0, k mod 2, 0] = 1; L_0[0, Dw-1, 0] = 1,
//          R_N[0, 0, 0] = 1 (the MPO's boundary vectors select its last /
//          first channel); right environments built from the right end;
//   bond (k, k+1): psi = A_k A_{k+1}; lowest eigenpair of H_eff(L_k, W, W,
//          R_{k+2}) by Lanczos from psi; trunc_svd(psi, 2, 1, chi_max, 0,
//          s_min); left-to-right: A_k = U, A_{k+1} = S V^T, L_{k+1} updated;
//          right-to-left: A_{k+1} = V^T, A_k = U S, R_{k+1} updated;
//   a sweep runs k = 0..N-2 then N-2..0; its energy is the last Ritz value.
#include <string.h>

#include <map>
#include <vector>

#include "heff_plan.cuh"

namespace {


tci_status contract3(tci_context ctx, tci_tensor a, const char* la, tci_tensor b, const char* lb, const char* lc,
                     tci_tensor* out) {
  *out = nullptr;
  return tci_contract(ctx, a, la, b, lb, out, lc);
}

// L'[b, w', b'] = sum A[a, s, b] L[a, w, a'] W[w, w', s, t] A[a', t, b']
tci_status update_left(tci_context ctx, tci_tensor L, tci_tensor A, tci_tensor W, tci_tensor* out) {
  TciOwned t1, t2;
  TCI_TRY(contract3(ctx, L, "awx", A, "xty", "awty", &t1.t));
  TCI_TRY(contract3(ctx, t1.t, "awty", W, "wvst", "avsy", &t2.t));
  return contract3(ctx, A, "asb", t2.t, "avsy", "bvy", out);
}

// R'[a, w, a'] = sum A[a, s, b] W[w, w', s, t] R[b, w', b'] A[a', t, b']
tci_status update_right(tci_context ctx, tci_tensor R, tci_tensor A, tci_tensor W, tci_tensor* out) {
  TciOwned t1, t2;
  TCI_TRY(contract3(ctx, R, "bvy", A, "xty", "bvxt", &t1.t));
  TCI_TRY(contract3(ctx, t1.t, "bvxt", W, "wvst", "bwsx", &t2.t));
  return contract3(ctx, A, "asb", t2.t, "bwsx", "awx", out);
}

tci_status unit_tensor(tci_context ctx, const int64_t* shape, int64_t flat_one, tci_tensor* out) {
  TCI_TRY(tci_zeros(ctx, TCI_F64, 3, shape, out));
  const double one = 1.0;
  TCI_CUDA(ctx, cudaMemcpyAsync((double*)(*out)->data + flat_one, &one, sizeof(double), cudaMemcpyHostToDevice,
                                ctx->stream));
  return TCI_OK;
}

}  // namespace

extern "C" tci_status tci_dmrg(tci_context ctx, tci_tensor W, int nsites, int64_t chi_max, int nsweeps,
                               int lanczos_steps, double s_min, double* energies, double* max_trunc_err) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "dmrg");
  if (!tci_ten_ok(W) || W->dtype != TCI_F64 || W->order != 4 || W->shape[2] != 2 || W->shape[3] != 2 ||
      W->shape[0] != W->shape[1] || !tci_is_rowmajor(W))
    return tci_fail(ctx, TCI_ERR_SHAPE, "dmrg: W must be a row-major F64 [Dw, Dw, 2, 2] tensor");
  if (nsites < 2 || chi_max < 1 || nsweeps < 1 || lanczos_steps < 1 || !energies)
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "dmrg: need nsites >= 2, chi_max >= 1, nsweeps >= 1, lanczos_steps >= 1");
  const int N = nsites;
  const int64_t Dw = W->shape[0];
  vs.info = "N=" + std::to_string(N) + " chi_max=" + std::to_string(chi_max);
  std::vector<TciOwned> A(N), L(N + 1), R(N + 2);
  const int64_t site_shape[3] = {1, 2, 1};
  for (int k = 0; k < N; ++k) TCI_TRY(unit_tensor(ctx, site_shape, k % 2, &A[k].t));
  const int64_t env_shape[3] = {1, Dw, 1};
  TCI_TRY(unit_tensor(ctx, env_shape, Dw - 1, &L[0].t));
  TCI_TRY(unit_tensor(ctx, env_shape, 0, &R[N].t));
  for (int k = N - 1; k >= 1; --k) TCI_TRY(update_right(ctx, R[k + 1].t, A[k].t, W, &R[k].t));

  // one H_eff plan per bond shape (chiL, chiR), reloaded with each bond's
  // environments: the MPO is the same everywhere, so W.W is computed once per
  // plan, and the plan's Lanczos graph is replayed from its third solve on
  std::map<std::pair<int64_t, int64_t>, tci_heff_plan> plans;
  struct PlanCache {
    std::map<std::pair<int64_t, int64_t>, tci_heff_plan>& m;
    ~PlanCache() {
      for (auto& kv : m) tci_heff_plan_destroy(&kv.second);
    }
  } plan_cache{plans};
  auto solve = [&](int k, tci_tensor* ground, double* theta) -> tci_status {
    TciOwned psi, x;
    TCI_TRY(contract3(ctx, A[k].t, "abc", A[k + 1].t, "cde", "abde", &psi.t));
    TCI_TRY(tci_allocate(ctx, TCI_F64, 4, psi.t->shape, &x.t));
    const auto key = std::make_pair(L[k].t->shape[0], R[k + 2].t->shape[0]);
    auto it = plans.find(key);
    if (it == plans.end()) {
      tci_heff_plan plan = nullptr;
      TCI_TRY(tci_heff_plan_create(ctx, L[k].t, W, R[k + 2].t, &plan));
      it = plans.emplace(key, plan).first;
    } else {
      // same_mpo = true skips the W.W recompute: valid because this driver applies
      // one MPO tensor W on every site (a per-site MPO would need false here)
      TCI_TRY(tci_heff_plan_reload_impl(it->second, L[k].t, W, W, R[k + 2].t, true));
    }
    int done = 0;
    TCI_TRY(tci_lanczos(it->second, psi.t, lanczos_steps, 1, theta, nullptr, nullptr, &done, x.t));
    *ground = x.release();
    return TCI_OK;
  };
  for (int sw = 0; sw < nsweeps; ++sw) {
    double theta = 0.0, terr_max = 0.0;
    for (int dir = 0; dir < 2; ++dir) {
      for (int step = 0; step < N - 1; ++step) {
        const int k = dir == 0 ? step : N - 2 - step;
        TciOwned x, u, s, vt, sd;
        TCI_TRY(solve(k, &x.t, &theta));
        double terr = 0.0;
        TCI_TRY(tci_trunc_svd(ctx, x.t, 2, &u.t, &s.t, &vt.t, &terr, 1, chi_max, 0.0, s_min));
        terr_max = terr > terr_max ? terr : terr_max;
        TCI_TRY(tci_diag_to(ctx, s.t, &sd.t));
        if (dir == 0) {
          tci_tensor next = nullptr;
          TCI_TRY(contract3(ctx, sd.t, "ab", vt.t, "bcd", "acd", &next));
          A[k + 1].reset(next);
          A[k].reset(u.release());
          tci_tensor ln = nullptr;
          TCI_TRY(update_left(ctx, L[k].t, A[k].t, W, &ln));
          L[k + 1].reset(ln);
        } else {
          tci_tensor prev = nullptr;
          TCI_TRY(contract3(ctx, u.t, "abc", sd.t, "cd", "abd", &prev));
          A[k].reset(prev);
          A[k + 1].reset(vt.release());
          tci_tensor rn = nullptr;
          TCI_TRY(update_right(ctx, R[k + 2].t, A[k + 1].t, W, &rn));
          R[k + 1].reset(rn);
        }
      }
    }
    energies[sw] = theta;
    if (max_trunc_err) max_trunc_err[sw] = terr_max;
  }
  return tci_synchronize(ctx);
}
