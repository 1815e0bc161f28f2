// Autotuner and plan cache for the split-BF16 tensor-core GEMM.
//
// Tuned per plan on the plan's own operands, timed with CUDA events on the
// context stream:
//   chunk_k  in {128, 256, 512} (<= the caller's accuracy cap; the hi*hi
//            accumulation error grows linearly with it, ~2.9e-8 per 16 of
//            depth per GEMM, measured on B300),
//   xchunk_k in {1024, 4096},
//   raster   in {0 (m-fastest), 8, 16 (m-block groups, n-fastest inside)}
//            for plans whose GEMMs have many tiles per dimension,
//   bn       tile width in {128, 64} for grouped plans (narrow tiles for
//            problems of few columns: less padding, half the MMA work per tile).
// The candidates first run in turn for at least 250 ms (the clock settles
// under the power cap), then every candidate is timed over four rounds in
// alternating order and keeps its median (the best time would favour whichever
// candidates ran while the GPU was cool).  Among the candidates within 2 % of the fastest the
// choice is stable: a grouped tile order (fewer DRAM re-reads), then the
// longer accumulation chunks (fewer drains), then the wider tile.
// Winners are cached in memory per (plan kind, shape, device) and, when the
// environment variable TCI_AUTOTUNE_CACHE names a file, appended to it as one
// line "key chunk_k xchunk_k raster bn ms"; a later process reads the file and
// reuses the entry without timing.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "heff_plan.cuh"

namespace {

std::mutex g_tune_mutex;
std::map<std::string, std::pair<tci_gemm_cfg, double>> g_tune_cache;
bool g_file_loaded = false;

void load_cache_file() {
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char* path = getenv("TCI_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[512];
  tci_gemm_cfg c;
  double ms = 0.0;
  while (fscanf(f, "%511s %d %d %d %d %lf", key, &c.chunk_k, &c.xchunk_k, &c.raster, &c.bn, &ms) == 6)
    g_tune_cache[key] = {c, ms};
  fclose(f);
}

void store_cache_file(const std::string& key, const tci_gemm_cfg& c, double ms) {
  const char* path = getenv("TCI_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %.6f\n", key.c_str(), c.chunk_k, c.xchunk_k, c.raster, c.bn, ms);
  fclose(f);
}

}  // namespace

tci_status tci_autotune(tci_context ctx, const std::string& key_in, int max_chunk_k, bool raster_candidates,
                        tci_status (*run)(void* arg, const tci_gemm_cfg& cfg), void* arg, tci_gemm_cfg* best,
                        double* best_ms, bool bn_candidates) {
  if (max_chunk_k < 128) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "autotune: max_chunk_k must be >= 128");
  cudaDeviceProp prop;
  TCI_CUDA(ctx, cudaGetDeviceProperties(&prop, ctx->device));
  std::string dev = prop.name;
  for (auto& ch : dev)
    if (ch == ' ') ch = '_';
  const std::string key = key_in + "|" + dev + "|cap" + std::to_string(max_chunk_k) + (bn_candidates ? "|bn" : "");
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_cache_file();
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *best = it->second.first;
      if (best_ms) *best_ms = it->second.second;
      return TCI_OK;
    }
  }
  std::vector<tci_gemm_cfg> cands;
  const int chunks[3] = {128, 256, 512};
  const int xchunks[2] = {1024, 4096};
  const int rasters[3] = {0, 8, 16};
  const int bns[2] = {128, 64};
  for (int c : chunks) {
    if (c > max_chunk_k) continue;
    for (int x : xchunks)
      for (int r : rasters) {
        if (!raster_candidates && r != 0) continue;
        for (int bn : bns) {
          if (!bn_candidates && bn != 128) continue;
          tci_gemm_cfg cfg;
          cfg.chunk_k = c;
          cfg.xchunk_k = x;
          cfg.raster = r;
          cfg.bn = bn;
          cands.push_back(cfg);
        }
      }
  }
  cudaEvent_t e0, e1;
  TCI_CUDA(ctx, cudaEventCreate(&e0));
  TCI_CUDA(ctx, cudaEventCreate(&e1));
  double bms = 1e300;
  tci_gemm_cfg bcfg = cands.front();
  tci_status s = TCI_OK;
  // The clock falls by 15-20 % while a GPU heats into its power cap, so the
  // candidates are first run in turn until at least kWarmMs of work has passed
  // (and at most 40 passes), then timed over four rounds in alternating
  // direction, and each candidate keeps the median of its rounds: a minimum
  // over rounds would favour whichever candidates ran while the GPU was cool.
  constexpr float kWarmMs = 250.f;
  std::vector<std::vector<double>> rounds(cands.size());
  float warm_total = 0.f;
  for (int pass = 0; pass < 40 && s == TCI_OK; ++pass) {   // warm-up (and kernel attributes)
    cudaEventRecord(e0, ctx->stream);
    for (const auto& cfg : cands)
      if ((s = run(arg, cfg)) != TCI_OK) break;
    cudaEventRecord(e1, ctx->stream);
    if (s != TCI_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = tci_cuda_fail(ctx, e, "autotune warm-up");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    warm_total += ms;
    if (warm_total >= kWarmMs) break;
  }
  for (int round = 0; round < 4 && s == TCI_OK; ++round) {
    for (size_t q = 0; q < cands.size() && s == TCI_OK; ++q) {
      const size_t i = (round & 1) ? cands.size() - 1 - q : q;
      float total = 0.f;
      const int reps = 3;
      cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < reps && s == TCI_OK; ++r) s = run(arg, cands[i]);
      cudaEventRecord(e1, ctx->stream);
      if (s != TCI_OK) break;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        s = tci_cuda_fail(ctx, e, "autotune timing");
        break;
      }
      cudaEventElapsedTime(&total, e0, e1);
      rounds[i].push_back((double)total / reps);
    }
  }
  std::vector<double> times(cands.size(), 1e300);
  for (size_t i = 0; i < cands.size(); ++i)
    if (!rounds[i].empty()) {
      std::vector<double> r = rounds[i];
      std::sort(r.begin(), r.end());
      times[i] = r.size() % 2 ? r[r.size() / 2] : 0.5 * (r[r.size() / 2 - 1] + r[r.size() / 2]);
    }
  double tmin = 1e300;
  for (size_t i = 0; i < cands.size() && s == TCI_OK; ++i) tmin = std::min(tmin, times[i]);
  // stable choice among the near-fastest: a grouped tile order (re-reads far fewer
  // operand bytes from DRAM, which the time hardly shows while the GEMM is
  // tensor-bound), then longer accumulation chunks, then the wider tile
  auto rank = [](const tci_gemm_cfg& c) {
    return std::make_tuple(c.raster == 16 ? 2 : c.raster == 8 ? 1 : 0, c.chunk_k, c.xchunk_k, c.bn);
  };
  for (size_t i = 0; i < cands.size() && s == TCI_OK; ++i)
    if (times[i] <= 1.02 * tmin && (bms == 1e300 || rank(cands[i]) > rank(bcfg))) {
      bms = times[i];
      bcfg = cands[i];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != TCI_OK) return s;
  TCI_TRY(tci_synchronize(ctx));
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = {bcfg, bms};
    store_cache_file(key, bcfg, bms);
  }
  *best = bcfg;
  if (best_ms) *best_ms = bms;
  return TCI_OK;
}

// ---------------------------------------------------------------- H_eff plans
namespace {
struct HeffTuneArg {
  tci_heff_plan p;
  const double* psi;
  double* out;
};

tci_status heff_run_cfg(void* a, const tci_gemm_cfg& cfg) {
  HeffTuneArg* t = (HeffTuneArg*)a;
  t->p->chunk_k = cfg.chunk_k;
  t->p->xchunk_k = cfg.xchunk_k;
  t->p->raster = cfg.raster;
  return tci_heff_apply_raw(t->p, t->psi, t->out, false);
}
}  // namespace

extern "C" tci_status tci_heff_autotune(tci_heff_plan p, tci_tensor psi, tci_tensor out, int max_chunk_k, int* chosen) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_autotune: invalid plan");
  if (p->cplx) return tci_fail(p->ctx, TCI_ERR_UNSUPPORTED, "heff_autotune: complex plans support tci_heff_apply only");
  tci_context ctx = p->ctx;
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "heff_autotune");
  if (!tci_ten_ok(psi) || !tci_ten_ok(out) || psi->dtype != TCI_F64 || out->dtype != TCI_F64 ||
      tci_numel(psi) != p->chiL * 4 * p->chiR || tci_numel(out) != p->chiL * 4 * p->chiR || !tci_is_rowmajor(psi) ||
      !tci_is_rowmajor(out))
    return tci_fail(ctx, TCI_ERR_SHAPE, "heff_autotune: psi/out must be row-major F64 [chiL,2,2,chiR]");
  if (p->prec == TCI_PREC_NATIVE) {   // nothing to tune on the FP64 path
    if (chosen) chosen[0] = chosen[1] = chosen[2] = 0;
    return TCI_OK;
  }
  HeffTuneArg arg{p, (const double*)psi->data, (double*)out->data};
  const std::string key = "heff|" + std::to_string(p->chiL) + "x" + std::to_string(p->chiR) + "|p" +
                          std::to_string(p->products);
  tci_gemm_cfg best;
  double ms = 0.0;
  TCI_TRY(tci_autotune(ctx, key, max_chunk_k, true, heff_run_cfg, &arg, &best, &ms));
  heff_run_cfg(&arg, best);   // leaves the plan configured with the winner (and U, V filled)
  float ww_ms = 0.f;
  TCI_TRY(tci_heff_tune_ww(p, &ww_ms));
  if (chosen) {
    chosen[0] = best.chunk_k;
    chosen[1] = best.xchunk_k;
    chosen[2] = best.raster;
  }
  vs.info = "chunk=" + std::to_string(best.chunk_k) + " xchunk=" + std::to_string(best.xchunk_k) +
            " raster=" + std::to_string(best.raster) + " ms=" + std::to_string(ms) + " ww_na=" + std::to_string(p->ww_na) +
            " ww_ms=" + std::to_string(ww_ms);
  return tci_synchronize(ctx);
}

extern "C" tci_status tci_heff_get_config(tci_heff_plan p, int* cfg) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_get_config: invalid plan");
  if (p->cplx) return tci_fail(p->ctx, TCI_ERR_UNSUPPORTED, "heff_get_config: complex plans support tci_heff_apply only");
  TCI_CHECK_CTX(p->ctx);
  if (!cfg) return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "heff_get_config: NULL cfg");
  const bool split = p->prec != TCI_PREC_NATIVE;
  cfg[0] = split ? p->chunk_k : 0;
  cfg[1] = split ? p->xchunk_k : 0;
  cfg[2] = split ? p->raster : 0;
  cfg[3] = split ? p->ww_na : 0;
  return TCI_OK;
}

extern "C" tci_status tci_heff_set_config(tci_heff_plan p, const int* cfg) {
  if (!p || p->magic != kPlanMagic) return tci_fail(nullptr, TCI_ERR_INVALID_ARG, "heff_set_config: invalid plan");
  if (p->cplx) return tci_fail(p->ctx, TCI_ERR_UNSUPPORTED, "heff_set_config: complex plans support tci_heff_apply only");
  TCI_CHECK_CTX(p->ctx);
  if (!cfg) return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "heff_set_config: NULL cfg");
  if (p->prec == TCI_PREC_NATIVE) return tci_fail(p->ctx, TCI_ERR_UNSUPPORTED, "heff_set_config: FP64 plan has no configuration");
  const int c = cfg[0], x = cfg[1], r = cfg[2], na = cfg[3];
  if (c < 32 || c % 32 != 0 || x < c || x % c != 0 || r < 0 || (na != 2 && na != 4))
    return tci_fail(p->ctx, TCI_ERR_INVALID_ARG, "heff_set_config: need 32 | chunk_k, chunk_k | xchunk_k, raster >= 0, W.W a' per thread 2 or 4");
  p->chunk_k = c;
  p->xchunk_k = x;
  p->raster = r;
  p->ww_na = na;
  return TCI_OK;
}
