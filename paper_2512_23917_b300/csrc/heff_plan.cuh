// H_eff plan object shared by the matvec and the Lanczos solver.
#pragma once

#include "tci_internal.cuh"

#define HEFF_DW 5
#define HEFF_NWW (HEFF_DW * 4 * HEFF_DW * 4)

constexpr int kPlanMagic = 0x4eff0001;

struct tci_heff_plan_s {
  int magic;
  tci_context ctx;
  int64_t chiL, chiR;
  tci_precision prec;
  int products;
  int chunk_k;     // split GEMM: K depth per hi*hi accumulation unit
  int xchunk_k;    // split GEMM: K depth per cross-product accumulation unit
  int raster = 0;  // split GEMM: tile order (autotuned)
  int ww_na = 4;      // split W.W kernel: a' per thread (2 or 4, autotuned)
  int vec_arith = 0;  // Lanczos vector arithmetic: 0 auto, 1 FP64, 2 double-float (FP32 pairs)
  int gs_mode = 0;    // Lanczos re-orthogonalisation: 0 DGKS second pass, 1 always twice
  // complex (C128) plan: owned copies of L, W, R and the contraction intermediates
  bool cplx = false;
  int64_t cd = 0, cDw = 0;
  tci_tensor cL = nullptr, cW = nullptr, cW2 = nullptr, cR = nullptr, cU[3] = {nullptr, nullptr, nullptr};
  tci_tensor cVin = nullptr, cVout = nullptr;   // borrowed views for the Lanczos matvec
  double ww[HEFF_NWW];   // WW[wl][s1 s2][wr][t1 t2]
  // intermediates
  void* U = nullptr;       // FP64 [(a',t1,t2), (b,wr)] (native) or FP32 U^T [(b,wr), (a',t1,t2)] (split)
  // native path
  double* L64 = nullptr;
  double* R64 = nullptr;
  double* V64 = nullptr;   // [(s1,s2,b), (wl,a')]
  // split path: bfloat16 piece planes [3][rows][Kp]
  int64_t Kp1 = 0, Kp2 = 0;
  void* Lp = nullptr;      // [3][chiL][Kp2]
  void* Rp = nullptr;      // [3][chiR*Dw][Kp1]
  void* psip = nullptr;    // [3][chiL*4][Kp1]
  void* Vp = nullptr;      // [3][4*chiR][Kp2]
  // host-buffer staging (copies overlapped with the compute on two copy streams)
  double* d_stage_in = nullptr;
  double* d_stage_out = nullptr;
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_in[8] = {}, ev_out[8] = {};
  // Lanczos workspace
  double* lz_V = nullptr;     // basis, capacity lz_cap vectors
  int lz_cap = 0;
  void* lz_Vs = nullptr;      // FP32 copy of the basis (hi planes, and lo planes with the double-float dots)
                              // capacity lz_vs_cap planes of ldv floats
  int lz_vs_cap = 0;
  double* lz_w = nullptr;
  double* lz_scal = nullptr;  // device scalars
  double* lz_part = nullptr;  // reduction partials
  double* lz_x64 = nullptr;   // double-float Lanczos with the FP64 matvec: matvec input / output
  double* lz_o64 = nullptr;
  int lz_stats[5] = {0, 0, 0, 0, 0};   // last tci_lanczos: steps, second GS passes, FP32-term passes,
                                       // double-float-term passes, fused pass 3
  // Lanczos solves replayed from a CUDA graph (real plans): the
  // launch sequence of a solve is fixed by its arguments (every branch is a
  // device gate), so a repeated call with the same key replays a captured
  // graph, its psi0 / x kernel arguments set for the call.
  void* ws = nullptr;          // FP64 plan: split-K partials of the matvec GEMMs
  size_t ws_bytes = 0;
  int lz_graphs = 1;
  int lz_last_graph = 0;       // the last solve ran as a graph launch (1) or eagerly (0)
  int64_t lz_graph_launches = 0;
  int lz_reduced = 1;   // reduced-precision small update terms (FP32 / double-float) allowed
  int lz_fuse = 0;      // split plans: first Gram-Schmidt projection formed in the matvec's GEMM2 (opt-in)
  int lz_shadow = 0;    // split plans, FP64 vectors: double-float Gram-Schmidt dots (opt-in; the
                        // first projection's from the basis's double-float shadow)
  tci_graph lz_graph;
  std::vector<int64_t> lz_graph_key, lz_last_key;
};

// out_mode 0: out is FP64; 2 (split precisions only): out is a normalised
// FP32 pair {hi, lo} per element.  psi_presplit: psi's bfloat16 pieces are
// already in p->psip (psi is then not read).
// Time the split W.W kernel variants on the plan's current intermediates and
// keep the faster (p->ww_na); *ms_out (may be NULL) receives its duration.
tci_status tci_heff_tune_ww(tci_heff_plan p, float* ms_out);
tci_status tci_heff_apply_complex_raw(tci_heff_plan p, const double* psi, double* out);
tci_status tci_heff_apply_raw(tci_heff_plan p, const double* psi, void* out, bool psi_presplit, int out_mode = 0);
// Split plan, psi pieces already in p->psip, FP64 out: the matvec with the
// dot products <V_i, out> (i < nv) and <out, out> formed in GEMM2's epilogue;
// part[i*part_stride + b], b < *grid, are the per-CTA partial sums.
tci_status tci_heff_apply_raw_dots(tci_heff_plan p, double* out, const double* V, int64_t ldv, int nv, double* part,
                                   int part_stride, int* grid);

// Reload environments of the same shapes into a real plan (see tci_heff_plan_reload);
// same_mpo skips recomputing W.W (the caller guarantees W and W2 are unchanged).
tci_status tci_heff_plan_reload_impl(tci_heff_plan p, tci_tensor L, tci_tensor W, tci_tensor W2, tci_tensor R,
                                     bool same_mpo);
