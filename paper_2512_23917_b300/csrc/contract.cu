// TCI "contract" (App. C.2; Sec. II.B.2: C_IJ = sum_S A_IS B_SJ).
//
// Planner: labels are classified into M (free in a), N (free in b), K
// (shared, summed) and batch (in a, b and c) groups; adjacent modes of a group that are contiguous with
// respect to each other in every tensor carrying them are coalesced.  When a
// group reduces to at most one mode per operand, the operand is read in place
// through its strides (no transpose is materialised); otherwise it is packed
// once (K8) into the canonical [M,K] / [N,K] layout.  Real contractions under
// a SPLIT precision pack directly into bfloat16 piece planes (K0) and run on
// the tcgen05 tensor cores.
#include <string.h>

#include <algorithm>
#include <vector>

#include "tci_internal.cuh"

namespace {

struct Mode {
  int64_t dim;
  int64_t sa, sb, sc;   // strides in a, b, c (0 where absent)
};

struct Group {
  std::vector<Mode> modes;
  int64_t size() const {
    int64_t n = 1;
    for (auto& m : modes) n *= m.dim;
    return n;
  }
};

// Merge mode i+1 into i when both are contiguous w.r.t. each other in all
// tensors that carry them (sX[i] == sX[i+1] * dim[i+1]); drop size-1 modes.
void coalesce(Group& g, bool use_a, bool use_b, bool use_c) {
  std::vector<Mode> out;
  for (auto& m : g.modes) {
    if (m.dim == 1) continue;
    if (!out.empty()) {
      Mode& p = out.back();
      bool ok = (!use_a || p.sa == m.sa * m.dim) && (!use_b || p.sb == m.sb * m.dim) && (!use_c || p.sc == m.sc * m.dim);
      if (ok) {
        p.dim *= m.dim;
        p.sa = m.sa;
        p.sb = m.sb;
        p.sc = m.sc;
        continue;
      }
    }
    out.push_back(m);
  }
  g.modes = out;
}

bool ranges_overlap(const tci_tensor_s* x, const tci_tensor_s* y) {
  if (!x->data || !y->data) return false;
  auto extent = [](const tci_tensor_s* t) {
    int64_t e = 1;
    for (int i = 0; i < t->order; ++i)
      if (t->shape[i] > 0) e += (t->shape[i] - 1) * t->strides[i];
    return e * (int64_t)tci_elem_bytes(t->dtype);
  };
  const char* a0 = (const char*)x->data;
  const char* b0 = (const char*)y->data;
  return a0 < b0 + extent(y) && b0 < a0 + extent(x);
}

}  // namespace

// Core: c_data (row-major over c's labels in the order given, or the strides
// given) = contract(a, b).  la/lb/lc are int labels.
static tci_status contract_impl(tci_context ctx, tci_tensor a, const int32_t* la, tci_tensor b, const int32_t* lb,
                                tci_tensor* pc, const int32_t* lc, int nc) {
  if (!tci_ten_ok(a) || !tci_ten_ok(b) || !pc) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "contract: invalid tensor argument");
  if (nc < 0 || nc > TCI_MAX_ORDER) return tci_fail(ctx, TCI_ERR_LABEL, "contract: %d output labels", nc);
  if ((a->order && !la) || (b->order && !lb) || (nc && !lc)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "contract: NULL label list");
  if (a->dtype != b->dtype) return tci_fail(ctx, TCI_ERR_DTYPE, "contract: operand dtypes differ");
  const tci_dtype dt = a->dtype;
  auto find = [](const int32_t* l, int n, int32_t v) {
    for (int i = 0; i < n; ++i)
      if (l[i] == v) return i;
    return -1;
  };
  for (int i = 0; i < a->order; ++i)
    if (find(la, i, la[i]) >= 0) return tci_fail(ctx, TCI_ERR_LABEL, "contract: label repeated within operand a");
  for (int i = 0; i < b->order; ++i)
    if (find(lb, i, lb[i]) >= 0) return tci_fail(ctx, TCI_ERR_LABEL, "contract: label repeated within operand b");
  for (int i = 0; i < nc; ++i)
    if (find(lc, i, lc[i]) >= 0) return tci_fail(ctx, TCI_ERR_LABEL, "contract: label repeated within c");

  int64_t cshape[TCI_MAX_ORDER];
  for (int i = 0; i < nc; ++i) {
    int ia = find(la, a->order, lc[i]), ib = find(lb, b->order, lc[i]);
    if (ia < 0 && ib < 0) return tci_fail(ctx, TCI_ERR_LABEL, "contract: output label not found in a or b");
    if (ia >= 0 && ib >= 0 && a->shape[ia] != b->shape[ib])
      return tci_fail(ctx, TCI_ERR_LABEL, "contract: bond dimension mismatch on a batch label");
    cshape[i] = ia >= 0 ? a->shape[ia] : b->shape[ib];
  }
  Group gm, gn, gk, gb;
  // K group (shared, not in c) in a's bond order; dims must agree
  for (int i = 0; i < a->order; ++i) {
    int ib = find(lb, b->order, la[i]);
    if (ib >= 0) {
      if (a->shape[i] != b->shape[ib]) return tci_fail(ctx, TCI_ERR_LABEL, "contract: bond dimension mismatch on a shared label");
      if (find(lc, nc, la[i]) < 0) gk.modes.push_back({a->shape[i], a->strides[i], b->strides[ib], 0});
    } else if (find(lc, nc, la[i]) < 0) {
      return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "contract: free label of a missing from c");
    }
  }
  for (int i = 0; i < b->order; ++i)
    if (find(la, a->order, lb[i]) < 0 && find(lc, nc, lb[i]) < 0)
      return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "contract: free label of b missing from c");

  // ----- output tensor
  tci_tensor c = *pc;
  int64_t cstr_rm[TCI_MAX_ORDER];
  tci_rowmajor_strides(nc, cshape, cstr_rm);
  bool reuse = false;   // write straight into the caller's borrowed c
  if (c) {
    if (!tci_ten_ok(c)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "contract: invalid output tensor");
    bool same = c->dtype == dt && c->order == nc;
    for (int i = 0; same && i < nc; ++i) same = c->shape[i] == cshape[i];
    bool aliases = ranges_overlap(c, a) || ranges_overlap(c, b);
    if (!c->alloc && c->data) {
      if (!same) return tci_fail(ctx, same ? TCI_ERR_SHAPE : (c->dtype != dt ? TCI_ERR_DTYPE : TCI_ERR_SHAPE),
                                 "contract: borrowed output has the wrong shape or dtype");
      reuse = !aliases;
    } else {
      reuse = same && !aliases && c->data != nullptr;
    }
  }
  const int64_t* cstr = reuse ? c->strides : cstr_rm;

  for (int i = 0; i < nc; ++i) {
    int ia = find(la, a->order, lc[i]);
    int ib = find(lb, b->order, lc[i]);
    if (ia >= 0 && ib >= 0) gb.modes.push_back({a->shape[ia], a->strides[ia], b->strides[ib], cstr[i]});
    else if (ia >= 0) gm.modes.push_back({a->shape[ia], a->strides[ia], 0, cstr[i]});
    else gn.modes.push_back({b->shape[ib], 0, b->strides[ib], cstr[i]});
  }
  coalesce(gm, true, false, true);
  coalesce(gn, false, true, true);
  coalesce(gk, true, true, false);
  coalesce(gb, true, true, true);
  const int64_t M = gm.size(), N = gn.size(), K = gk.size(), NB = gb.size();
  int64_t numel_c = 1;
  for (int i = 0; i < nc; ++i) numel_c *= cshape[i];

  // result storage
  void* cdata = reuse ? c->data : nullptr;
  void* cnew = nullptr;
  if (!reuse) {
    TCI_TRY(tci_dev_alloc(ctx, (size_t)numel_c * tci_elem_bytes(dt), &cnew));
    cdata = cnew;
  }
  std::vector<void*> scratch;
  auto cleanup = [&](tci_status s) {
    if (!scratch.empty()) cudaStreamSynchronize(ctx->stream);
    for (void* p : scratch) tci_dev_free(p);
    if (s != TCI_OK && cnew) tci_dev_free(cnew);
    return s;
  };
  const size_t eb = tci_elem_bytes(dt);

  if (!gb.modes.empty()) {
    // ----- batch bonds (labels in a, b and c): one product per batch slice.
    // Operands are packed to [batch][M][K] and [batch][N][K], the slices run
    // as one launch -- the native-arithmetic batched GEMM, or for real
    // operands under a split precision one grouped split-BF16 tensor-core
    // launch with a problem per slice -- and the [batch][M][N] result is
    // scattered into c.
    if (NB * M * N > 0) {
      auto pack3 = [&](tci_tensor t, bool is_a, const Group& g1, void** out) -> tci_status {
        int ord = 0;
        int64_t shp[3 * TCI_MAX_ORDER], str[3 * TCI_MAX_ORDER];
        const Group* gs[3] = {&gb, &g1, &gk};
        for (const Group* g : gs)
          for (auto& m : g->modes) {
            shp[ord] = m.dim;
            str[ord] = is_a ? m.sa : m.sb;   // not t == a: a and b may be one tensor
            ++ord;
          }
        if (ord > TCI_MAX_ORDER) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "contract: too many non-coalescible modes");
        TCI_TRY(tci_dev_alloc(ctx, (size_t)(NB * g1.size() * K) * eb, out));
        scratch.push_back(*out);
        if (ord == 0) {   // every bond of size 1: a single element
          TCI_CUDA(ctx, cudaMemcpyAsync(*out, t->data, eb, cudaMemcpyDeviceToDevice, ctx->stream));
          return TCI_OK;
        }
        return tci_launch_permute_copy(ctx, dt, ord, shp, t->data, str, *out);
      };
      void *Apk = nullptr, *Bpk = nullptr, *Ck = nullptr;
      tci_status s = TCI_OK;
      if (K > 0) {
        s = pack3(a, true, gm, &Apk);
        if (s == TCI_OK) s = pack3(b, false, gn, &Bpk);
      }
      if (s == TCI_OK) s = tci_dev_alloc(ctx, (size_t)(NB * M * N) * eb, &Ck);
      if (s != TCI_OK) return cleanup(s);
      scratch.push_back(Ck);
      const bool split = ctx->precision != TCI_PREC_NATIVE && (dt == TCI_F64 || dt == TCI_F32);
      if (K == 0) {
        cudaMemsetAsync(Ck, 0, (size_t)(NB * M * N) * eb, ctx->stream);
      } else if (split) {
        // pieces of all slices in one plane set each: [3][NB*M][Kp] and [3][NB*N][Kp]
        const int64_t Kp = (K + 7) / 8 * 8;
        void *Ap3 = nullptr, *Bp3 = nullptr;
        s = tci_dev_alloc(ctx, (size_t)(3 * NB * M * Kp) * 2, &Ap3);
        if (s == TCI_OK) {
          scratch.push_back(Ap3);
          s = tci_dev_alloc(ctx, (size_t)(3 * NB * N * Kp) * 2, &Bp3);
        }
        if (s == TCI_OK) {
          scratch.push_back(Bp3);
          s = tci_launch_split3(ctx, dt, Apk, NB * M, K, K, 1, Ap3, Kp);
        }
        if (s == TCI_OK) s = tci_launch_split3(ctx, dt, Bpk, NB * N, K, K, 1, Bp3, Kp);
        std::vector<tci_split_problem> probs;
        for (int64_t bi = 0; bi < NB && s == TCI_OK; ++bi) {
          tci_split_problem q;
          q.Ap = (const char*)Ap3 + (size_t)(bi * M * Kp) * 2;
          q.Bp = (const char*)Bp3 + (size_t)(bi * N * Kp) * 2;
          q.M = M;
          q.N = N;
          q.Kp = Kp;
          q.C = (char*)Ck + (size_t)(bi * M * N) * eb;
          q.out_mode = dt == TCI_F64 ? 0 : 1;
          q.scm = N;
          q.scn = 1;
          q.a_plane_rows = NB * M;
          q.b_plane_rows = NB * N;
          probs.push_back(q);
        }
        tci_split_group* grp = nullptr;
        if (s == TCI_OK) s = tci_split_group_create(ctx, (int)probs.size(), probs.data(), &grp);
        if (s == TCI_OK)
          s = tci_split_group_launch(ctx, grp, ctx->precision == TCI_PREC_SPLIT_BF16_3 ? 3 : 6, ctx->split_chunk_k,
                                     ctx->split_xchunk_k, 0);
        if (grp) tci_split_group_destroy(grp);
      } else {
        s = tci_gemm_native_batched(ctx, dt, NB, M, N, K, Apk, M * K, K, 1, Bpk, N * K, K, 1, Ck, M * N, N, 1);
      }
      if (s != TCI_OK) return cleanup(s);
      int ord = 0;
      int64_t shp[3 * TCI_MAX_ORDER], sst[3 * TCI_MAX_ORDER], dst[3 * TCI_MAX_ORDER];
      const Group* gs[3] = {&gb, &gm, &gn};
      for (const Group* g : gs)
        for (auto& m : g->modes) {
          shp[ord] = m.dim;
          dst[ord] = m.sc;
          ++ord;
        }
      tci_rowmajor_strides(ord, shp, sst);
      s = tci_launch_strided_copy(ctx, dt, ord, shp, Ck, sst, cdata, dst);
      if (s != TCI_OK) return cleanup(s);
    }
  } else if (M * N > 0 && K == 0) {
    // K == 0 (a shared bond of dimension 0): c = 0
    if (reuse && !tci_is_rowmajor(c)) {
      // zero through a strided scatter of a zero buffer
      void* z = nullptr;
      tci_status s = tci_dev_alloc(ctx, (size_t)numel_c * eb, &z);
      if (s != TCI_OK) return cleanup(s);
      scratch.push_back(z);
      cudaMemsetAsync(z, 0, (size_t)numel_c * eb, ctx->stream);
      s = tci_launch_strided_copy(ctx, dt, nc, cshape, z, cstr_rm, c->data, c->strides);
      if (s != TCI_OK) return cleanup(s);
    } else {
      cudaMemsetAsync(cdata, 0, (size_t)numel_c * eb, ctx->stream);
    }
  } else if (M * N > 0) {
    // ----- operand views: in place when each group has <= 1 mode
    auto pack = [&](tci_tensor t, const int32_t* lt, const Group& g1, const Group& g2, bool g1_is_m, const void** ptr,
                    int64_t* s1, int64_t* s2) -> tci_status {
      // operand element (x1, x2), x1 over g1 (m or n), x2 over k
      bool direct = g1.modes.size() <= 1 && g2.modes.size() <= 1;
      if (direct) {
        *ptr = t->data;
        *s1 = g1.modes.empty() ? 0 : (g1_is_m ? g1.modes[0].sa : g1.modes[0].sb);
        *s2 = g2.modes.empty() ? 0 : (g1_is_m ? g2.modes[0].sa : g2.modes[0].sb);
        return TCI_OK;
      }
      // pack [g1 modes..., g2 modes...] row-major
      int ord = 0;
      int64_t shp[2 * TCI_MAX_ORDER], str[2 * TCI_MAX_ORDER];
      for (auto& m : g1.modes) { shp[ord] = m.dim; str[ord] = (g1_is_m ? m.sa : m.sb); ++ord; }
      for (auto& m : g2.modes) { shp[ord] = m.dim; str[ord] = (g1_is_m ? m.sa : m.sb); ++ord; }
      if (ord > TCI_MAX_ORDER) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "contract: too many non-coalescible modes");
      void* p = nullptr;
      TCI_TRY(tci_dev_alloc(ctx, (size_t)(g1.size() * g2.size()) * eb, &p));
      scratch.push_back(p);
      TCI_TRY(tci_launch_permute_copy(ctx, dt, ord, shp, t->data, str, p));
      *ptr = p;
      *s1 = g2.size();
      *s2 = 1;
      (void)lt;
      (void)g1_is_m;
      return TCI_OK;
    };
    const void* Ap;
    const void* Bp;
    int64_t sam, sak, sbn, sbk;
    tci_status s = pack(a, la, gm, gk, true, &Ap, &sam, &sak);
    if (s != TCI_OK) return cleanup(s);
    s = pack(b, lb, gn, gk, false, &Bp, &sbn, &sbk);
    if (s != TCI_OK) return cleanup(s);

    // ----- output view
    void* Cp = cdata;
    int64_t scm, scn;
    bool cdirect = gm.modes.size() <= 1 && gn.modes.size() <= 1;
    if (cdirect) {
      scm = gm.modes.empty() ? 0 : gm.modes[0].sc;
      scn = gn.modes.empty() ? 0 : gn.modes[0].sc;
    } else {
      void* p = nullptr;
      s = tci_dev_alloc(ctx, (size_t)(M * N) * eb, &p);
      if (s != TCI_OK) return cleanup(s);
      scratch.push_back(p);
      Cp = p;
      scm = N;
      scn = 1;
    }
    const bool real = dt == TCI_F32 || dt == TCI_F64;
    if (real && ctx->precision != TCI_PREC_NATIVE) {
      // K0 split/pack into piece planes, then the tcgen05 GEMM (FP64 result)
      int64_t Kp = (K + 7) / 8 * 8;
      void *Apc = nullptr, *Bpc = nullptr;
      s = tci_dev_alloc(ctx, (size_t)3 * M * Kp * 2, &Apc);
      if (s != TCI_OK) return cleanup(s);
      scratch.push_back(Apc);
      s = tci_dev_alloc(ctx, (size_t)3 * N * Kp * 2, &Bpc);
      if (s != TCI_OK) return cleanup(s);
      scratch.push_back(Bpc);
      s = tci_launch_split3(ctx, dt, Ap, M, K, sam, sak, Apc, Kp);
      if (s == TCI_OK) s = tci_launch_split3(ctx, dt, Bp, N, K, sbn, sbk, Bpc, Kp);
      if (s != TCI_OK) return cleanup(s);
      const int products = ctx->precision == TCI_PREC_SPLIT_BF16_3 ? 3 : 6;
      s = tci_gemm_split_bf16(ctx, M, N, Kp, Apc, Bpc, Cp, dt == TCI_F32 ? 1 : 0, scm, scn, products,
                              ctx->split_chunk_k, ctx->split_xchunk_k, 0);
      if (s != TCI_OK) return cleanup(s);
    } else {
      s = tci_gemm_native(ctx, dt, M, N, K, Ap, sam, sak, Bp, sbn, sbk, Cp, scm, scn);
      if (s != TCI_OK) return cleanup(s);
    }
    if (!cdirect) {
      // scatter [M modes..., N modes...] into c's strides
      int ord = 0;
      int64_t shp[2 * TCI_MAX_ORDER], sst[2 * TCI_MAX_ORDER], dst[2 * TCI_MAX_ORDER];
      for (auto& m : gm.modes) { shp[ord] = m.dim; dst[ord] = m.sc; ++ord; }
      for (auto& m : gn.modes) { shp[ord] = m.dim; dst[ord] = m.sc; ++ord; }
      if (ord > TCI_MAX_ORDER) return cleanup(tci_fail(ctx, TCI_ERR_UNSUPPORTED, "contract: too many output modes"));
      tci_rowmajor_strides(ord, shp, sst);
      s = tci_launch_strided_copy(ctx, dt, ord, shp, Cp, sst, cdata, dst);
      if (s != TCI_OK) return cleanup(s);
    }
  }
  TCI_TRY(cleanup(TCI_OK));

  // ----- place the result
  if (reuse) return TCI_OK;
  if (!c) {
    tci_tensor t = new tci_tensor_s();
    t->magic = kTenMagic;
    t->dtype = dt;
    t->order = nc;
    for (int i = 0; i < nc; ++i) {
      t->shape[i] = cshape[i];
      t->strides[i] = cstr_rm[i];
    }
    t->data = cnew;
    t->alloc = cnew;
    t->device = ctx->device;
    *pc = t;
    return TCI_OK;
  }
  if (!c->alloc && c->data) {
    // borrowed output that aliased an operand: copy the result into it
    tci_status s = tci_launch_strided_copy(ctx, dt, nc, cshape, cnew, cstr_rm, c->data, c->strides);
    cudaStreamSynchronize(ctx->stream);
    tci_dev_free(cnew);
    return s;
  }
  // owned (or empty) output: adopt the new storage
  cudaStreamSynchronize(ctx->stream);
  tci_dev_free(c->alloc);
  c->alloc = cnew;
  c->data = cnew;
  c->dtype = dt;
  c->order = nc;
  for (int i = 0; i < nc; ++i) {
    c->shape[i] = cshape[i];
    c->strides[i] = cstr_rm[i];
  }
  return TCI_OK;
}

extern "C" tci_status tci_contract_l(tci_context ctx, tci_tensor a, const int32_t* labels_a, tci_tensor b,
                                     const int32_t* labels_b, tci_tensor* c, const int32_t* labels_c, int nc) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "contract");
  if (ctx->verbose && tci_ten_ok(a) && tci_ten_ok(b)) vs.info = tci_shape_str(a) + " x " + tci_shape_str(b);
  return contract_impl(ctx, a, labels_a, b, labels_b, c, labels_c, nc);
}

extern "C" tci_status tci_contract(tci_context ctx, tci_tensor a, const char* labels_a, tci_tensor b,
                                   const char* labels_b, tci_tensor* c, const char* labels_c) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "contract");
  if (!labels_a || !labels_b || !labels_c) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "contract: NULL label string");
  if (!tci_ten_ok(a) || !tci_ten_ok(b)) return tci_fail(ctx, TCI_ERR_INVALID_ARG, "contract: invalid tensor argument");
  if (ctx->verbose) vs.info = std::string(labels_a) + "," + labels_b + "->" + labels_c + " " + tci_shape_str(a) + " x " + tci_shape_str(b);
  int na = (int)strlen(labels_a), nb = (int)strlen(labels_b), nc = (int)strlen(labels_c);
  if (na != a->order || nb != b->order)
    return tci_fail(ctx, TCI_ERR_LABEL, "contract: label string length differs from tensor order");
  if (nc > TCI_MAX_ORDER) return tci_fail(ctx, TCI_ERR_LABEL, "contract: too many output labels");
  int32_t ia[TCI_MAX_ORDER], ib[TCI_MAX_ORDER], ic[TCI_MAX_ORDER];
  for (int i = 0; i < na; ++i) ia[i] = (unsigned char)labels_a[i];
  for (int i = 0; i < nb; ++i) ib[i] = (unsigned char)labels_b[i];
  for (int i = 0; i < nc; ++i) ic[i] = (unsigned char)labels_c[i];
  return contract_impl(ctx, a, ia, b, ib, c, ic, nc);
}
