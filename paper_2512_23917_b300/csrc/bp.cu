// Belief propagation on the norm network of a tensor-network state (App. B),
// driven from the host through the library's batched contraction.
//
// Every directed bond i -> j carries a message M_{i->j}[b, b'] (ket, bra
// bond index).  One synchronous iteration forms, for every message,
//
//   M_{i->j} = sum_s V_i[s, .., b, ..] V_i[s, .., b', ..] prod_{k != j} M_{k->i}
//
// then normalises it to unit Frobenius norm.  Messages whose sites have the
// same shape and leave through the same bond position form one group; a
// group is one batched contraction chain over a batch bond z:
//
//   T_0 = V[z, s, a, b, c];  T_q = T_{q-1} x M_q[z, q, Q] (bond q -> Q), q != out
//   R[z, o, O] = T_last x V[z, s, A, B, C]  (summed over s and the bra bonds)
//
// All messages live in two device arenas (current, next); a gather kernel
// stacks each group's incoming messages, and a normalise kernel writes the
// group's results into the next arena together with ||M_new - M_old||_F.
#include <algorithm>
#include <map>
#include <vector>

#include "tci_internal.cuh"

namespace {

constexpr int kBpT = 256;
constexpr int kMaxDegree = 6;   // site order 1 + k plus the batch bond <= 8
const char kKet[] = "abcdef";
const char kBra[] = "ABCDEF";

// dst[b][i] = arena[offs[b] + i]
__global__ void k_gather_off(const double* __restrict__ arena, const int64_t* __restrict__ offs, int64_t len,
                             double* __restrict__ dst) {
  const int64_t b = blockIdx.y;
  const double* src = arena + offs[b];
  double* d = dst + b * len;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = src[i];
}

// dst[b][i] = srcs[b][i]
__global__ void k_gather_ptr(const double* const* __restrict__ srcs, int64_t len, double* __restrict__ dst) {
  const int64_t b = blockIdx.y;
  const double* src = srcs[b];
  double* d = dst + b * len;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = src[i];
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kBpT / 32; ++k) t += red[k];
    red[kBpT / 32] = t;
  }
  __syncthreads();
  t = red[kBpT / 32];
  __syncthreads();
  return t;
}

// One block per message b: next[offs[b] + i] = raw[b][i] / ||raw[b]||,
// res[b] = ||next - cur|| over the message (a zero message stays zero).
__global__ void __launch_bounds__(kBpT) k_normalise(const double* __restrict__ raw, int64_t len,
                                                    const int64_t* __restrict__ offs, const double* __restrict__ cur,
                                                    double* __restrict__ next, double* __restrict__ res) {
  __shared__ double red[kBpT / 32 + 1];
  const int64_t b = blockIdx.x;
  const double* r = raw + b * len;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < len; i += kBpT) s = fma(r[i], r[i], s);
  const double nrm = sqrt(block_sum(s, red));
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  const double* c = cur + offs[b];
  double* n = next + offs[b];
  double d2 = 0.0;
  for (int64_t i = threadIdx.x; i < len; i += kBpT) {
    const double v = r[i] * inv;
    n[i] = v;
    const double dv = v - c[i];
    d2 = fma(dv, dv, d2);
  }
  d2 = block_sum(d2, red);
  if (threadIdx.x == 0) res[b] = sqrt(d2);
}

struct Group {
  std::vector<int64_t> shape;   // site shape (d, chi_1 .. chi_k)
  int out = 0;                  // outgoing bond position
  std::vector<int> site;        // per member: site index
  std::vector<int> msg;         // per member: outgoing message index
  std::vector<std::vector<int>> in;   // per bond q: incoming message index per member
  // device data
  double* vstack = nullptr;
  std::vector<double*> mstack;  // per bond q (nullptr for q == out)
  std::vector<int64_t*> in_offs;
  int64_t* out_offs = nullptr;
  double* res = nullptr;        // device residual slots (into a shared array)
  int res_base = 0;
  TciOwned V;                    // wraps vstack as [B, d, chi..]
  std::vector<TciOwned> M;       // wraps mstack[q] as [B, chi_q, chi_q]
  std::vector<TciOwned> T;       // contraction intermediates (reused)
  TciOwned R;                    // [B, chi_out, chi_out]
};

unsigned grid_x(tci_context ctx, int64_t len, int64_t batch) {
  int64_t bx = (len + kBpT - 1) / kBpT;
  const int64_t want = std::max<int64_t>(1, (int64_t)ctx->num_sms * 8 / std::max<int64_t>(1, batch));
  return (unsigned)std::max<int64_t>(1, std::min(bx, want));
}

}  // namespace

extern "C" tci_status tci_bp(tci_context ctx, int nsites, int nedges, const int64_t* edges, const tci_tensor* sites,
                             tci_tensor* messages, int niters, double tol, int* iters_done, double* residuals) {
  TCI_CHECK_CTX(ctx);
  TciVerboseScope vs(ctx, "bp");
  if (iters_done) *iters_done = 0;
  if (nsites < 0 || nedges < 0 || niters < 0 || (nedges > 0 && (!edges || !messages)) || (nsites > 0 && !sites))
    return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bp: invalid graph or buffers");
  // neighbour lists: (neighbour, incoming message) sorted by neighbour
  std::vector<std::vector<std::pair<int, int>>> nb(nsites);
  for (int e = 0; e < nedges; ++e) {
    const int64_t u = edges[2 * e], v = edges[2 * e + 1];
    if (u < 0 || v < 0 || u >= nsites || v >= nsites || u == v)
      return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bp: edge %d (%lld, %lld) out of range or a loop", e, (long long)u,
                      (long long)v);
    nb[u].push_back({(int)v, 2 * e + 1});
    nb[v].push_back({(int)u, 2 * e});
  }
  for (int i = 0; i < nsites; ++i) {
    std::sort(nb[i].begin(), nb[i].end());
    for (size_t q = 1; q < nb[i].size(); ++q)
      if (nb[i][q].first == nb[i][q - 1].first)
        return tci_fail(ctx, TCI_ERR_INVALID_ARG, "bp: repeated edge between %d and %d", i, nb[i][q].first);
    if ((int)nb[i].size() > kMaxDegree)
      return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "bp: site %d has degree %zu (at most %d)", i, nb[i].size(), kMaxDegree);
    const tci_tensor V = sites[i];
    if (!tci_ten_ok(V) || V->dtype != TCI_F64 || !tci_is_rowmajor(V))
      return tci_fail(ctx, TCI_ERR_DTYPE, "bp: site %d must be a row-major F64 tensor", i);
    if (V->order != 1 + (int)nb[i].size())
      return tci_fail(ctx, TCI_ERR_SHAPE, "bp: site %d has order %d, expected 1 + degree = %zu", i, V->order,
                      1 + nb[i].size());
  }
  // message shapes and arena offsets
  const int nmsg = 2 * nedges;
  std::vector<int64_t> off(nmsg + 1, 0), chi(nmsg, 0);
  for (int e = 0; e < nedges; ++e) {
    const int u = (int)edges[2 * e], v = (int)edges[2 * e + 1];
    int qu = 0, qv = 0;
    while (nb[u][qu].first != v) ++qu;
    while (nb[v][qv].first != u) ++qv;
    const int64_t cu = sites[u]->shape[1 + qu], cv = sites[v]->shape[1 + qv];
    if (cu != cv) return tci_fail(ctx, TCI_ERR_SHAPE, "bp: bond dimensions of edge %d differ (%lld, %lld)", e,
                                  (long long)cu, (long long)cv);
    for (int m : {2 * e, 2 * e + 1}) {
      const tci_tensor M = messages[m];
      if (!tci_ten_ok(M) || M->dtype != TCI_F64 || !tci_is_rowmajor(M) || M->order != 2 || M->shape[0] != cu ||
          M->shape[1] != cu)
        return tci_fail(ctx, TCI_ERR_SHAPE, "bp: message %d must be a row-major F64 [%lld, %lld] tensor", m,
                        (long long)cu, (long long)cu);
      chi[m] = cu;
    }
  }
  for (int m = 0; m < nmsg; ++m) off[m + 1] = off[m] + chi[m] * chi[m];
  vs.info = "sites=" + std::to_string(nsites) + " messages=" + std::to_string(nmsg);
  if (nmsg == 0 || niters == 0) return tci_synchronize(ctx);

  // groups of messages with the same site shape and outgoing bond position
  std::map<std::pair<std::vector<int64_t>, int>, int> key_of;
  std::vector<Group> groups;
  for (int i = 0; i < nsites; ++i) {
    std::vector<int64_t> shape(sites[i]->shape, sites[i]->shape + sites[i]->order);
    for (int q = 0; q < (int)nb[i].size(); ++q) {
      const auto key = std::make_pair(shape, q);
      auto it = key_of.find(key);
      if (it == key_of.end()) {
        it = key_of.emplace(key, (int)groups.size()).first;
        groups.emplace_back();
        groups.back().shape = shape;
        groups.back().out = q;
        groups.back().in.resize(nb[i].size());
      }
      Group& g = groups[it->second];
      g.site.push_back(i);
      // the message leaving i towards nb[i][q] is the one that enters nb[i][q] from i
      const int j = nb[i][q].first;
      int mo = -1;
      for (auto& pr : nb[j])
        if (pr.first == i) mo = pr.second;
      g.msg.push_back(mo);
      for (int k = 0; k < (int)nb[i].size(); ++k) g.in[k].push_back(k == q ? -1 : nb[i][k].second);
    }
  }

  // device buffers
  std::vector<void*> bufs;
  auto alloc = [&](size_t bytes, void** p) -> tci_status {
    TCI_TRY(tci_dev_alloc(ctx, bytes, p));
    bufs.push_back(*p);
    return TCI_OK;
  };
  struct Cleanup {
    tci_context ctx;
    std::vector<void*>* bufs;
    ~Cleanup() {
      for (void* p : *bufs) tci_dev_free(p);
    }
  } cleanup{ctx, &bufs};
  double *arena[2] = {nullptr, nullptr}, *res_all = nullptr;
  TCI_TRY(alloc(sizeof(double) * off[nmsg], (void**)&arena[0]));
  TCI_TRY(alloc(sizeof(double) * off[nmsg], (void**)&arena[1]));
  TCI_TRY(alloc(sizeof(double) * nmsg, (void**)&res_all));
  for (int m = 0; m < nmsg; ++m)
    TCI_CUDA(ctx, cudaMemcpyAsync(arena[0] + off[m], messages[m]->data, sizeof(double) * chi[m] * chi[m],
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  int res_base = 0;
  for (Group& g : groups) {
    const int64_t B = (int64_t)g.site.size();
    const int k = (int)g.shape.size() - 1;
    if (B > 65535) return tci_fail(ctx, TCI_ERR_UNSUPPORTED, "bp: more than 65535 messages of one kind");
    int64_t vlen = 1;
    for (int64_t x : g.shape) vlen *= x;
    TCI_TRY(alloc(sizeof(double) * B * vlen, (void**)&g.vstack));
    std::vector<const double*> ptrs(B);
    for (int64_t b = 0; b < B; ++b) ptrs[b] = (const double*)sites[g.site[b]]->data;
    const double** dptrs = nullptr;
    TCI_TRY(alloc(sizeof(double*) * B, (void**)&dptrs));
    TCI_CUDA(ctx, cudaMemcpyAsync(dptrs, ptrs.data(), sizeof(double*) * B, cudaMemcpyHostToDevice, ctx->stream));
    k_gather_ptr<<<dim3(grid_x(ctx, vlen, B), (unsigned)B), kBpT, 0, ctx->stream>>>(dptrs, vlen, g.vstack);
    TCI_CUDA(ctx, cudaGetLastError());
    int64_t vshape[TCI_MAX_ORDER];
    vshape[0] = B;
    for (int q = 0; q <= k; ++q) vshape[1 + q] = g.shape[q];
    TCI_TRY(tci_tensor_wrap(ctx, TCI_F64, k + 2, vshape, nullptr, g.vstack, &g.V.t));
    g.mstack.assign(k, nullptr);
    g.in_offs.assign(k, nullptr);
    g.M.resize(k);
    g.T.resize(k);
    for (int q = 0; q < k; ++q) {
      if (q == g.out) continue;
      const int64_t c = g.shape[1 + q];
      TCI_TRY(alloc(sizeof(double) * B * c * c, (void**)&g.mstack[q]));
      std::vector<int64_t> o(B);
      for (int64_t b = 0; b < B; ++b) o[b] = off[g.in[q][b]];
      TCI_TRY(alloc(sizeof(int64_t) * B, (void**)&g.in_offs[q]));
      TCI_CUDA(ctx, cudaMemcpyAsync(g.in_offs[q], o.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice, ctx->stream));
      const int64_t mshape[3] = {B, c, c};
      TCI_TRY(tci_tensor_wrap(ctx, TCI_F64, 3, mshape, nullptr, g.mstack[q], &g.M[q].t));
    }
    std::vector<int64_t> o(B);
    for (int64_t b = 0; b < B; ++b) o[b] = off[g.msg[b]];
    TCI_TRY(alloc(sizeof(int64_t) * B, (void**)&g.out_offs));
    TCI_CUDA(ctx, cudaMemcpyAsync(g.out_offs, o.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice, ctx->stream));
    g.res_base = res_base;
    g.res = res_all + res_base;
    res_base += (int)B;
  }
  // host copies of the pointer/offset tables must outlive the async uploads
  TCI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));

  std::vector<double> res_host(nmsg);
  int cur = 0, it = 0;
  for (; it < niters; ++it) {
    for (Group& g : groups) {
      const int64_t B = (int64_t)g.site.size();
      const int k = (int)g.shape.size() - 1;
      // labels: z batch, s physical, ket a.., bra A..
      std::string lab = "zs";
      for (int q = 0; q < k; ++q) lab += kKet[q];
      tci_tensor T = g.V.t;
      for (int q = 0; q < k; ++q) {
        if (q == g.out) continue;
        const int64_t c = g.shape[1 + q];
        k_gather_off<<<dim3(grid_x(ctx, c * c, B), (unsigned)B), kBpT, 0, ctx->stream>>>(arena[cur], g.in_offs[q],
                                                                                         c * c, g.mstack[q]);
        TCI_CUDA(ctx, cudaGetLastError());
        std::string next = lab;
        next[2 + q] = kBra[q];
        const std::string ml = std::string("z") + kKet[q] + kBra[q];
        TCI_TRY(tci_contract(ctx, T, lab.c_str(), g.M[q].t, ml.c_str(), &g.T[q].t, next.c_str()));
        T = g.T[q].t;
        lab = next;
      }
      std::string bra = "zs";
      for (int q = 0; q < k; ++q) bra += kBra[q];
      const std::string ol = std::string("z") + kKet[g.out] + kBra[g.out];
      TCI_TRY(tci_contract(ctx, T, lab.c_str(), g.V.t, bra.c_str(), &g.R.t, ol.c_str()));
      const int64_t c = g.shape[1 + g.out];
      k_normalise<<<(unsigned)B, kBpT, 0, ctx->stream>>>((const double*)g.R.t->data, c * c, g.out_offs, arena[cur],
                                                         arena[1 - cur], g.res);
      TCI_CUDA(ctx, cudaGetLastError());
    }
    TCI_CUDA(ctx, cudaMemcpyAsync(res_host.data(), res_all, sizeof(double) * nmsg, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    TCI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double r = 0.0;
    for (double x : res_host) r = std::max(r, x);
    if (residuals) residuals[it] = r;
    cur = 1 - cur;
    if (r <= tol) {
      ++it;
      break;
    }
  }
  if (iters_done) *iters_done = it;
  for (int m = 0; m < nmsg; ++m)
    TCI_CUDA(ctx, cudaMemcpyAsync(messages[m]->data, arena[cur] + off[m], sizeof(double) * chi[m] * chi[m],
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  return tci_synchronize(ctx);
}
