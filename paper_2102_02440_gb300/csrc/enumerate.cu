// Join-order enumeration over sketch estimates (Sec. 5, Algorithm 1): for every join graph,
// a depth-first search over left-deep orders that follow the graph's edges, from every
// source vertex in increasing f(v) = alpha card(v) / max card + beta deg(v) / max deg,
// extending a prefix by its neighbours in increasing estimate of the extended sub-plan,
// pruning a prefix whose cost exceeds the best complete plan's, and ending a source's
// search after max_plans complete plans.
//
// Cost of a plan: the sum of the estimates of its join prefixes of two or more tables (the
// first table adds nothing).  Ties: sources and candidates by table id.  A NaN estimate
// (beyond the exact range) counts as +inf, a negative one as 0.  Pruning and the update of
// the best plan are strict, so of equal-cost plans the first found is kept.
//
// One warp per graph, its first lane searching: the search is sequential (each source's
// search starts from the best cost found so far), and graphs in separate warps do not
// serialise each other's divergent paths.  The stack, one frame per prefix length, lives in
// the workspace; the estimates come from the device array the estimate wrote (no host round
// trip), found through the graph's open-addressing table of sub-plan masks.  f(v) and the
// costs are computed with explicitly rounded double operations (no fused multiply-add), so
// every comparison sees the same values as a plain IEEE evaluation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace cmpk {
namespace {

constexpr int kEnumMaxN = CMP_MAX_TABLES;  // 64

struct EnumGraph {
  int32_t n, h_log2;            // tables; log2 of its hash table's slots
  int64_t h_begin, n_masks;     // its hash table in the slot array; its sub-plans
  const int64_t* card;          // device [n]: exact selected counts
  uint64_t adj[kEnumMaxN];
  int32_t deg[kEnumMaxN];
};
// One slot of a graph's table: a sub-plan mask (0 = empty; masks are nonzero) and the
// index of its estimate.  Linear probing from enum_hash(mask); at most half the slots used.
struct EnumSlot {
  uint64_t mask;
  int64_t sub;
};
__host__ __device__ inline uint64_t enum_hash(uint64_t m) {
  m ^= m >> 31;
  m *= 0x7fb5d329728ea185ull;
  m ^= m >> 27;
  m *= 0x81dadef4bc2dd44dull;
  return m ^ (m >> 33);
}

struct EnumPlanHdr {
  uint64_t magic;
  int32_t version, n_graphs;
  int64_t n_sub, n_slots;
  int64_t off_graphs, off_slots, total_bytes, ws_bytes;
};
constexpr uint64_t kEnumPlanMagic = 0x434d50454e554d31ull;  // "CMPENUM1"

// One search frame per prefix length: the prefix, its cost, its candidates sorted by
// (estimate, id) with their estimates, the next candidate, the neighbours of the prefix.
struct EnumFrames {
  uint64_t mask[kEnumMaxN];
  uint64_t nb[kEnumMaxN];
  double cost[kEnumMaxN];
  int32_t n_cand[kEnumMaxN], next[kEnumMaxN], path[kEnumMaxN];
  uint8_t cand[kEnumMaxN][kEnumMaxN];
  double e[kEnumMaxN][kEnumMaxN];
};
constexpr size_t kEnumFrameBytes = (sizeof(EnumFrames) + 255) & ~size_t(255);

struct EnumArgs {
  const EnumGraph* graphs;
  const EnumSlot* slots;
  const double* est;
  int32_t n_graphs;
  double alpha, beta;
  int64_t max_plans, max_nodes;
  unsigned char* ws;
  int32_t* order;
  double* cost;
  int64_t* stats;
  int32_t* status;
};

__device__ double lookup(const EnumArgs& A, const EnumGraph& g, uint64_t m, bool* missing) {
  const uint64_t size = uint64_t(1) << g.h_log2;
  uint64_t i = enum_hash(m) & (size - 1);
  int64_t sub = -1;
  for (uint64_t probe = 0; probe < size; probe++) {  // the table has empty slots: ends early
    const EnumSlot sl = A.slots[g.h_begin + int64_t(i)];
    if (sl.mask == m) {
      sub = sl.sub;
      break;
    }
    if (sl.mask == 0) break;
    i = (i + 1) & (size - 1);
  }
  if (sub < 0) {
    *missing = true;
    return INFINITY;
  }
  const double v = A.est[sub];
  if (v != v) return INFINITY;  // NaN: beyond the exact range
  return v < 0.0 ? 0.0 : v;
}

// Candidates of frame d: neighbours of the prefix not in it, sorted by (estimate, id).
__device__ void expand(const EnumArgs& A, const EnumGraph& g, EnumFrames& F, int d, bool* missing) {
  const uint64_t m = F.mask[d];
  uint64_t c = F.nb[d] & ~m;
  int k = 0;
  while (c) {
    const int v = __ffsll(static_cast<long long>(c)) - 1;
    c &= c - 1;
    const double e = lookup(A, g, m | (1ull << v), missing);
    int j = k;  // ids ascend, so inserting after equal estimates keeps id order
    while (j > 0 && F.e[d][j - 1] > e) {
      F.e[d][j] = F.e[d][j - 1];
      F.cand[d][j] = F.cand[d][j - 1];
      j--;
    }
    F.e[d][j] = e;
    F.cand[d][j] = uint8_t(v);
    k++;
  }
  F.n_cand[d] = k;
  F.next[d] = 0;
}

}  // namespace

__global__ void k_enumerate(const __grid_constant__ EnumArgs A) {
  const int gi = int(blockIdx.x);
  if (gi >= A.n_graphs || threadIdx.x != 0) return;
  const EnumGraph& g = A.graphs[gi];
  EnumFrames& F = *reinterpret_cast<EnumFrames*>(A.ws + size_t(gi) * kEnumFrameBytes);
  const int n = g.n;
  const uint64_t full = n == 64 ? ~0ull : ((1ull << n) - 1);
  // source order: f(v) increasing, ties by id
  int64_t mc = 0;
  int32_t md = 0;
  for (int v = 0; v < n; v++) {
    mc = max(mc, g.card[v]);
    md = max(md, g.deg[v]);
  }
  int src[kEnumMaxN];
  double fv[kEnumMaxN];
  for (int v = 0; v < n; v++) {
    const double a = mc > 0 ? __ddiv_rn(__ll2double_rn(g.card[v]), __ll2double_rn(mc)) : 0.0;
    const double b = md > 0 ? __ddiv_rn(double(g.deg[v]), double(md)) : 0.0;
    const double f = __dadd_rn(__dmul_rn(A.alpha, a), __dmul_rn(A.beta, b));
    int j = v;
    while (j > 0 && fv[j - 1] > f) {
      fv[j] = fv[j - 1];
      src[j] = src[j - 1];
      j--;
    }
    fv[j] = f;
    src[j] = v;
  }
  double min_cost = INFINITY;
  int best[kEnumMaxN];
  bool have = false, missing = false, out_of_budget = false;
  int64_t plans = 0, nodes = 0, pruned = 0;
  for (int si = 0; si < n && !out_of_budget; si++) {
    const int s = src[si];
    int64_t p = 0;
    F.mask[0] = 1ull << s;
    F.nb[0] = g.adj[s];
    F.cost[0] = 0.0;
    F.path[0] = s;
    if (F.mask[0] == full) {  // one table: the plan is complete and costs nothing
      plans++;
      if (0.0 < min_cost) {
        min_cost = 0.0;
        best[0] = s;
        have = true;
      }
      continue;
    }
    expand(A, g, F, 0, &missing);
    int d = 0;
    while (d >= 0) {
      if (F.next[d] == F.n_cand[d]) {
        d--;
        continue;
      }
      const int k = F.next[d]++;
      const int v = F.cand[d][k];
      if (nodes == A.max_nodes) {  // budget spent: stop after exactly max_nodes extensions
        out_of_budget = true;
        break;
      }
      nodes++;
      const uint64_t cm = F.mask[d] | (1ull << v);
      const double cc = __dadd_rn(F.cost[d], F.e[d][k]);
      F.path[d + 1] = v;
      if (cc > min_cost) {  // early pruning
        pruned++;
        continue;
      }
      if (cm == full) {  // complete plan
        plans++;
        if (cc < min_cost) {
          min_cost = cc;
          for (int t = 0; t <= d + 1; t++) best[t] = F.path[t];
          have = true;
        }
        if (A.max_plans > 0 && ++p == A.max_plans) break;  // this source's search ends (-1: never)
        continue;
      }
      d++;
      F.mask[d] = cm;
      F.nb[d] = F.nb[d - 1] | g.adj[v];
      F.cost[d] = cc;
      expand(A, g, F, d, &missing);
    }
  }
  for (int t = 0; t < kEnumMaxN; t++) A.order[int64_t(gi) * kEnumMaxN + t] = (have && t < n) ? best[t] : -1;
  A.cost[gi] = have ? min_cost : INFINITY;
  A.stats[int64_t(gi) * 3 + 0] = plans;
  A.stats[int64_t(gi) * 3 + 1] = nodes;
  A.stats[int64_t(gi) * 3 + 2] = pruned;
  if (missing) set_status(A.status, CMP_EUNSUPPORTED);
  if (out_of_budget) set_status(A.status, CMP_ETIMEOUT);
}

namespace {

struct EnumPlanParts {
  std::vector<EnumGraph> graphs;
  std::vector<EnumSlot> slots;
  EnumPlanHdr hdr;
};

cmp_status enum_plan(const cmp_graph* graphs, int32_t n_graphs, int32_t n_sub, const int32_t* sub_graph,
                     const uint64_t* sub_mask, EnumPlanParts* P) {
  if (!graphs || n_graphs < 1 || n_sub < 0 || (n_sub && (!sub_graph || !sub_mask))) return CMP_EINVAL;
  P->graphs.assign(size_t(n_graphs), EnumGraph{});
  std::vector<std::vector<std::pair<uint64_t, int64_t>>> per(n_graphs);
  for (int32_t q = 0; q < n_sub; q++) {
    const int32_t gi = sub_graph[q];
    if (gi < 0 || gi >= n_graphs || sub_mask[q] == 0) return CMP_EINVAL;
    const int32_t nt = graphs[gi].n_tables;
    if (nt < 64 && (sub_mask[q] >> nt) != 0) return CMP_EINVAL;
    per[gi].push_back({sub_mask[q], q});
  }
  P->slots.clear();
  for (int32_t gi = 0; gi < n_graphs; gi++) {
    const cmp_graph& cg = graphs[gi];
    if (cg.n_tables < 1 || cg.n_tables > kEnumMaxN || cg.n_edges < 0 || !cg.survivors_dev) return CMP_EINVAL;
    if (cg.n_edges && (!cg.edge_u || !cg.edge_v)) return CMP_EINVAL;
    EnumGraph& g = P->graphs[gi];
    std::memset(&g, 0, sizeof(g));
    g.n = cg.n_tables;
    g.card = cg.survivors_dev;
    for (int32_t e = 0; e < cg.n_edges; e++) {
      const int u = cg.edge_u[e], v = cg.edge_v[e];
      if (u < 0 || u >= g.n || v < 0 || v >= g.n || u == v) return CMP_EINVAL;
      g.adj[u] |= 1ull << v;
      g.adj[v] |= 1ull << u;
      g.deg[u]++;
      g.deg[v]++;
    }
    auto& list = per[gi];
    std::sort(list.begin(), list.end());
    for (size_t i = 1; i < list.size(); i++)
      if (list[i].first == list[i - 1].first) return CMP_EINVAL;  // one estimate per sub-plan
    g.n_masks = int64_t(list.size());
    int lg = 4;
    while ((int64_t(1) << lg) < 2 * g.n_masks) lg++;
    g.h_log2 = lg;
    g.h_begin = int64_t(P->slots.size());
    P->slots.resize(P->slots.size() + (size_t(1) << lg), EnumSlot{0, 0});
    EnumSlot* tab = P->slots.data() + g.h_begin;
    const uint64_t size = uint64_t(1) << lg;
    for (const auto& x : list) {
      uint64_t i = enum_hash(x.first) & (size - 1);
      while (tab[i].mask != 0) i = (i + 1) & (size - 1);
      tab[i] = EnumSlot{x.first, x.second};
    }
  }
  EnumPlanHdr& H = P->hdr;
  std::memset(&H, 0, sizeof(H));
  H.magic = kEnumPlanMagic;
  H.version = 2;
  H.n_graphs = n_graphs;
  H.n_sub = n_sub;
  H.n_slots = int64_t(P->slots.size());
  size_t off = align16(sizeof(EnumPlanHdr));
  H.off_graphs = int64_t(off);
  off += align16(sizeof(EnumGraph) * P->graphs.size());
  H.off_slots = int64_t(off);
  off += align16(sizeof(EnumSlot) * P->slots.size());
  H.total_bytes = int64_t(off);
  H.ws_bytes = int64_t(kEnumFrameBytes * size_t(n_graphs));
  return CMP_OK;
}

}  // namespace
}  // namespace cmpk

using namespace cmpk;

extern "C" {

cmp_status cmp_enum_plan_bytes(const cmp_graph* graphs, int32_t n_graphs, int32_t n_sub, const int32_t* sub_graph,
                               const uint64_t* sub_mask, size_t* plan_bytes, size_t* ws_bytes) {
  if (!plan_bytes || !ws_bytes) return CMP_EINVAL;
  EnumPlanParts P;
  const cmp_status st = enum_plan(graphs, n_graphs, n_sub, sub_graph, sub_mask, &P);
  if (st != CMP_OK) return st;
  *plan_bytes = size_t(P.hdr.total_bytes);
  *ws_bytes = size_t(P.hdr.ws_bytes);
  return CMP_OK;
}

cmp_status cmp_enum_plan_encode(const cmp_graph* graphs, int32_t n_graphs, int32_t n_sub, const int32_t* sub_graph,
                                const uint64_t* sub_mask, void* plan_host, size_t plan_bytes) {
  if (!plan_host) return CMP_EINVAL;
  EnumPlanParts P;
  const cmp_status st = enum_plan(graphs, n_graphs, n_sub, sub_graph, sub_mask, &P);
  if (st != CMP_OK) return st;
  if (plan_bytes < size_t(P.hdr.total_bytes)) return CMP_EWORKSPACE;
  unsigned char* b = static_cast<unsigned char*>(plan_host);
  std::memset(b, 0, size_t(P.hdr.total_bytes));
  std::memcpy(b, &P.hdr, sizeof(P.hdr));
  std::memcpy(b + P.hdr.off_graphs, P.graphs.data(), sizeof(EnumGraph) * P.graphs.size());
  if (!P.slots.empty()) std::memcpy(b + P.hdr.off_slots, P.slots.data(), sizeof(EnumSlot) * P.slots.size());
  return CMP_OK;
}

cmp_status cmp_enumerate(const void* plan_host, const void* plan_dev, const double* est_dev, const cmp_enum_cfg* cfg,
                         void* ws_dev, size_t ws_bytes, int32_t* order_dev, double* cost_dev, int64_t* stats_dev,
                         int32_t* status_dev, void* stream) {
  if (!plan_host || !plan_dev) return CMP_EINVAL;
  EnumPlanHdr H;
  std::memcpy(&H, plan_host, sizeof(H));
  if (H.magic != kEnumPlanMagic || H.version != 2) return CMP_EINVAL;
  if (!order_dev || !cost_dev || !stats_dev || (H.n_sub > 0 && !est_dev)) return CMP_EINVAL;
  if (!ws_dev || ws_bytes < size_t(H.ws_bytes)) return CMP_EWORKSPACE;
  double alpha = 0.5, beta = 0.5;
  int64_t max_plans = 10, max_nodes = int64_t(1) << 26;
  if (cfg) {
    if (!(cfg->alpha >= 0.0) || !(cfg->beta >= 0.0) || cfg->max_plans < -1 || cfg->max_nodes < 0) return CMP_EINVAL;
    if (cfg->alpha != 0.0 || cfg->beta != 0.0) alpha = cfg->alpha, beta = cfg->beta;
    if (cfg->max_plans != 0) max_plans = cfg->max_plans;  // -1: no limit
    if (cfg->max_nodes > 0) max_nodes = cfg->max_nodes;
  }
  const unsigned char* pd = static_cast<const unsigned char*>(plan_dev);
  EnumArgs a;
  a.graphs = reinterpret_cast<const EnumGraph*>(pd + H.off_graphs);
  a.slots = reinterpret_cast<const EnumSlot*>(pd + H.off_slots);
  a.est = est_dev;
  a.n_graphs = H.n_graphs;
  a.alpha = alpha;
  a.beta = beta;
  a.max_plans = max_plans;
  a.max_nodes = max_nodes;
  a.ws = static_cast<unsigned char*>(ws_dev);
  a.order = order_dev;
  a.cost = cost_dev;
  a.stats = stats_dev;
  a.status = status_dev;
  k_enumerate<<<unsigned(H.n_graphs), 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? CMP_OK : CMP_ECUDA;
}

}  // extern "C"
