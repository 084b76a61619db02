// C ABI: presort and the batched sub-plan estimate (host planning + launches).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "estimate.cuh"

using namespace cmpk;

namespace {

struct EstShape {
  int32_t threads, ctas_per_sm, cond_chunk, flags;
};

cmp_status est_shape(const cmp_estimate_cfg* cfg, EstShape* s) {
  s->threads = (cfg && cfg->threads > 0) ? cfg->threads : 1024;
  s->ctas_per_sm = (cfg && cfg->ctas_per_sm > 0) ? cfg->ctas_per_sm : 1;
  s->cond_chunk = (cfg && cfg->cond_chunk > 0) ? cfg->cond_chunk : 64;
  s->flags = cfg ? cfg->flags : 0;
  if (s->flags & ~int32_t(CMP_EST_GENERIC_ONLY)) return CMP_EINVAL;
  if (s->threads < 32 || s->threads > 1024 || s->threads % 32 || s->ctas_per_sm > 32) return CMP_EINVAL;
  return CMP_OK;
}

struct PlanOut {
  std::vector<EstSub> subs;
  std::vector<EstOp> ops;
  std::vector<EstIn> ins;
  std::vector<EstItem> items;
  int32_t max_slots = 0, max_in = 1, max_suf = 0, max_rank = 0;
  std::vector<TriSub> tris;
  std::vector<EstItem> tri_items;  // appended after the generic items
  int32_t tri_max_leaves = 0;
};

bool graph_ok(const cmp_graph& g) {
  if (g.n_tables < 1 || g.n_tables > CMP_MAX_TABLES || g.n_edges < 0) return false;
  if (g.n_edges && (!g.edge_u || !g.edge_v || !g.sketch || !g.abs_sorted || !g.perm || !g.ranks || !g.slot))
    return false;
  if (!g.survivors_dev) return false;
  if (g.sample_rate)
    for (int t = 0; t < g.n_tables; t++)
      if (!(g.sample_rate[t] >= 0.0 && g.sample_rate[t] <= 1.0)) return false;  // NaN fails too
  for (int e = 0; e < g.n_edges; e++) {
    if (g.edge_u[e] < 0 || g.edge_u[e] >= g.n_tables || g.edge_v[e] < 0 || g.edge_v[e] >= g.n_tables) return false;
    if (g.edge_u[e] == g.edge_v[e]) return false;
    for (int end = 0; end < 2; end++)
      if (!g.sketch[2 * e + end] || !g.abs_sorted[2 * e + end] || !g.perm[2 * e + end] || !g.ranks[2 * e + end] ||
          g.slot[2 * e + end] < 0 || g.slot[2 * e + end] >= CMP_MAX_SKETCHES)
        return false;
  }
  return true;
}

// Triangle evaluation (estimate_tri.cu): the only cycle is a-W-b, closed by the
// conditioned edge a-b, and every other table is a leaf joined to a, b or W.  Returns
// false, leaving P unchanged, for any other shape.
bool plan_triangle(const cmp_graph& g, const std::vector<int>& es, const std::vector<char>& tree, int e_star,
                   uint64_t mask, int32_t d, int32_t w, int32_t sub_index, PlanOut* P, EstSub* sb) {
  const int nt = g.n_tables;
  const int a = g.edge_u[e_star], b = g.edge_v[e_star];
  auto touches = [&](int e, int t) { return g.edge_u[e] == t || g.edge_v[e] == t; };
  auto other = [&](int e, int t) { return g.edge_u[e] == t ? g.edge_v[e] : g.edge_u[e]; };
  auto end_of = [&](int e, int t) { return g.edge_u[e] == t ? 0 : 1; };
  int W = -1, eaW = -1, ebW = -1;
  for (int t = 0; t < nt && W < 0; t++) {
    if (!((mask >> t) & 1) || t == a || t == b) continue;
    int ea = -1, eb = -1;
    for (int e : es) {
      if (!tree[e] || !touches(e, t)) continue;
      if (other(e, t) == a) ea = e;
      if (other(e, t) == b) eb = e;
    }
    if (ea >= 0 && eb >= 0) {
      W = t;
      eaW = ea;
      ebW = eb;
    }
  }
  if (W < 0) return false;
  std::vector<int> deg(nt, 0);
  for (int e : es) deg[g.edge_u[e]]++, deg[g.edge_v[e]]++;
  for (int t = 0; t < nt; t++) {
    if (!((mask >> t) & 1) || t == a || t == b || t == W) continue;
    if (deg[t] != 1) return false;
    for (int e : es)
      if (touches(e, t) && other(e, t) != a && other(e, t) != b && other(e, t) != W) return false;
  }
  const int nodes[3] = {a, b, W};
  for (int n = 0; n < 3; n++)
    if (deg[nodes[n]] - 2 > kTriMaxLeaves) return false;
  TriSub ts;
  std::memset(&ts, 0, sizeof(ts));
  ts.sub = sub_index;
  int32_t leaves = 0;
  for (int n = 0; n < 3; n++) {
    const int t = nodes[n];
    TriNode& nd = ts.node[n];
    nd.in_begin = int32_t(P->ins.size());
    nd.k = 0;
    nd.ia = nd.ib = -1;
    for (int e : es) {  // ascending edge id
      if (!touches(e, t)) continue;
      const int me = end_of(e, t);
      EstIn x;
      std::memset(&x, 0, sizeof(x));
      x.s = g.sketch[2 * e + me];
      x.abs = g.abs_sorted[2 * e + me];
      x.perm = g.perm[2 * e + me];
      x.rk = g.ranks[2 * e + me];
      x.tslot = g.slot[2 * e + me];
      x.slot = x.suf = -1;
      if (e == e_star) {
        x.kind = kInCond;
      } else if (e == eaW || e == ebW) {
        x.kind = kInSlot;
      } else {
        x.kind = kInLeaf;
        x.msk = g.sketch[2 * e + end_of(e, other(e, t))];
      }
      if (e == (n == 1 ? ebW : eaW)) nd.ia = nd.k;
      if (e == (n == 2 ? ebW : e_star)) nd.ib = nd.k;
      P->ins.push_back(x);
      nd.k++;
    }
    leaves = std::max(leaves, nd.k - 2);
  }
  P->tri_max_leaves = std::max(P->tri_max_leaves, leaves);
  const int32_t nch = (w + kTriCols - 1) / kTriCols;
  sb->tri = int32_t(P->tris.size());
  sb->cond = 1;
  sb->n_ops = 0;
  sb->n_chunks = nch;
  sb->item_begin = int64_t(P->tri_items.size());  // offset by the generic items in plan_all
  P->tris.push_back(ts);
  for (int i = 0; i < d; i++)
    for (int ch = 0; ch < nch; ch++) {
      EstItem it;
      it.sub = sub_index;
      it.row = i;
      it.c0 = ch * kTriCols;
      it.c1 = std::min(w, (ch + 1) * kTriCols);
      P->tri_items.push_back(it);
    }
  return true;
}

// Plan one sub-plan: spanning tree by BFS from the lowest table id (edges in id order),
// non-tree edges conditioned, post-order operations for every non-leaf table.
cmp_status plan_sub(const cmp_graph& g, uint64_t mask, int32_t d, int32_t w, int32_t sub_index, int32_t chunk,
                    int32_t flags, PlanOut* P) {
  const int nt = g.n_tables;
  if (mask == 0 || (nt < 64 && (mask >> nt) != 0)) return CMP_EINVAL;
  std::vector<int> es;
  for (int e = 0; e < g.n_edges; e++)
    if (((mask >> g.edge_u[e]) & 1) && ((mask >> g.edge_v[e]) & 1)) es.push_back(e);
  int root = 0;
  while (!((mask >> root) & 1)) root++;
  std::vector<int> order{root}, parent_edge(nt, -1);
  std::vector<char> seen(nt, 0), tree(g.n_edges, 0);
  seen[root] = 1;
  for (size_t h = 0; h < order.size(); h++) {
    const int t = order[h];
    for (int e : es) {
      const int o = g.edge_u[e] == t ? g.edge_v[e] : (g.edge_v[e] == t ? g.edge_u[e] : -1);
      if (o < 0 || seen[o]) continue;
      seen[o] = 1;
      parent_edge[o] = e;
      tree[e] = 1;
      order.push_back(o);
    }
  }
  if (int(order.size()) != __builtin_popcountll(mask)) return CMP_EINVAL;  // not connected
  EstSub sb;
  std::memset(&sb, 0, sizeof(sb));
  sb.scale = 1.0;  // sampled tables: prod over the sub-plan's tables, ascending, of 1 / rate
  if (g.sample_rate)
    for (int t = 0; t < nt; t++) {
      const double r = g.sample_rate[t];
      if (((mask >> t) & 1) && r > 0.0 && r < 1.0) sb.scale = sb.scale * (1.0 / r);
    }
  sb.op_begin = int32_t(P->ops.size());
  sb.item_begin = int64_t(P->items.size());
  sb.tri = -1;
  if (order.size() == 1) {
    sb.single = 1;
    sb.sv = g.survivors_dev + root;
    P->subs.push_back(sb);
    return CMP_OK;
  }
  std::vector<int> cond;
  for (int e : es)
    if (!tree[e]) cond.push_back(e);
  if (cond.size() > 1) return CMP_EUNSUPPORTED;  // more than one independent cycle
  if (cond.size() == 1 && !(flags & CMP_EST_GENERIC_ONLY) && w <= kTriMaxW &&
      plan_triangle(g, es, tree, cond[0], mask, d, w, sub_index, P, &sb)) {
    P->subs.push_back(sb);
    return CMP_OK;
  }
  std::vector<int> deg(nt, 0);
  for (int e : es) deg[g.edge_u[e]]++, deg[g.edge_v[e]]++;
  auto is_leaf = [&](int t) { return t != root && deg[t] == 1; };
  auto end_of = [&](int e, int t) { return g.edge_u[e] == t ? 0 : 1; };
  std::vector<int> slot_of(nt, -1);
  std::vector<char> slot_busy;
  int32_t n_suf = 0;
  for (size_t h = order.size(); h-- > 0;) {
    const int t = order[h];
    if (is_leaf(t)) continue;
    EstOp op;
    std::memset(&op, 0, sizeof(op));
    op.k = 0;
    op.p = -1;
    op.out_slot = -1;
    op.in_begin = int32_t(P->ins.size());
    std::vector<int> consumed;
    for (int e : es) {
      if (g.edge_u[e] != t && g.edge_v[e] != t) continue;
      const int me = end_of(e, t);
      EstIn x;
      std::memset(&x, 0, sizeof(x));
      x.s = g.sketch[2 * e + me];
      x.abs = g.abs_sorted[2 * e + me];
      x.perm = g.perm[2 * e + me];
      x.rk = g.ranks[2 * e + me];
      x.tslot = g.slot[2 * e + me];
      x.suf = -1;
      if (e == parent_edge[t]) {
        x.kind = kInOutput;
        op.p = op.k;
      } else if (tree[e]) {
        x.suf = n_suf++;
        const int child = g.edge_u[e] == t ? g.edge_v[e] : g.edge_u[e];
        if (is_leaf(child)) {
          x.kind = kInLeaf;
          x.msk = g.sketch[2 * e + end_of(e, child)];
        } else {
          x.kind = kInSlot;
          x.slot = slot_of[child];
          consumed.push_back(slot_of[child]);
        }
      } else {
        x.kind = kInCond;
      }
      P->ins.push_back(x);
      op.k++;
    }
    if (op.p >= 0) {  // output slot: a free slot not read by this operation
      int s = -1;
      for (size_t q = 0; q < slot_busy.size(); q++)
        if (!slot_busy[q]) {
          s = int(q);
          break;
        }
      if (s < 0) {
        s = int(slot_busy.size());
        slot_busy.push_back(0);
      }
      slot_busy[s] = 1;
      op.out_slot = s;
      slot_of[t] = s;
    }
    for (int s : consumed) slot_busy[s] = 0;
    op.rank_off = 0;
    P->max_slots = std::max<int32_t>(P->max_slots, int32_t(slot_busy.size()));
    P->max_in = std::max<int32_t>(P->max_in, op.k);
    P->ops.push_back(op);
  }
  P->max_suf = std::max(P->max_suf, n_suf);
  sb.cond = cond.empty() ? 0 : 1;
  sb.n_ops = int32_t(P->ops.size()) - sb.op_begin;
  if (sb.n_ops > kEstMaxOps || int32_t(P->ins.size()) - P->ops[sb.op_begin].in_begin > kEstMaxSubIn)
    return CMP_EUNSUPPORTED;
  sb.n_chunks = cond.empty() ? 1 : (w + chunk - 1) / chunk;
  P->subs.push_back(sb);
  for (int i = 0; i < d; i++)
    for (int ch = 0; ch < sb.n_chunks; ch++) {
      EstItem it;
      it.sub = sub_index;
      it.row = i;
      it.c0 = cond.empty() ? 0 : ch * chunk;
      it.c1 = cond.empty() ? 1 : std::min(w, (ch + 1) * chunk);
      P->items.push_back(it);
    }
  return CMP_OK;
}

cmp_status plan_all(const cmp_graph* graphs, int32_t n_graphs, int32_t d, int32_t w, int32_t n_sub,
                    const int32_t* sub_graph, const uint64_t* sub_mask, const cmp_estimate_cfg* cfg, PlanOut* P,
                    EstPlanHdr* H) {
  if (!graphs || n_graphs < 1 || d < 1 || d > CMP_MAX_D || w < 1 || w > CMP_MAX_W || n_sub < 0) return CMP_EINVAL;
  EstShape shape;
  if (est_shape(cfg, &shape) != CMP_OK) return CMP_EINVAL;
  if (n_sub && (!sub_graph || !sub_mask)) return CMP_EINVAL;
  for (int32_t gi = 0; gi < n_graphs; gi++)
    if (!graph_ok(graphs[gi])) return CMP_EINVAL;
  for (int32_t q = 0; q < n_sub; q++) {
    if (sub_graph[q] < 0 || sub_graph[q] >= n_graphs) return CMP_EINVAL;
    const cmp_status st = plan_sub(graphs[sub_graph[q]], sub_mask[q], d, w, q, shape.cond_chunk, shape.flags, P);
    if (st != CMP_OK) return st;
  }
  // triangle items after the generic ones (the generic kernel runs [0, n_gen_items))
  const int64_t n_gen = int64_t(P->items.size());
  for (EstSub& sb : P->subs)
    if (sb.tri >= 0) sb.item_begin += n_gen;
  P->items.insert(P->items.end(), P->tri_items.begin(), P->tri_items.end());
  std::memset(H, 0, sizeof(*H));
  H->magic = kEstPlanMagic;
  H->version = kEstPlanVersion;
  H->d = d;
  H->w = w;
  H->max_slots = P->max_slots;
  H->max_in = P->max_in;
  H->threads = shape.threads;
  const int64_t cap = int64_t(sm_count()) * shape.ctas_per_sm;
  H->grid = int32_t(std::max<int64_t>(1, std::min<int64_t>(n_gen, cap)));
  H->n_gen_items = n_gen;
  H->n_tri = int64_t(P->tris.size());
  H->tri_max_leaves = P->tri_max_leaves;
  H->tri_nch = (w + kTriCols - 1) / kTriCols;
  H->tri_row_bytes = H->n_tri ? tri_layout(w, P->tri_max_leaves).bytes : 0;
  H->n_sub = n_sub;
  H->n_ops = int64_t(P->ops.size());
  H->n_in = int64_t(P->ins.size());
  H->n_items = int64_t(P->items.size());
  size_t off = align16(sizeof(EstPlanHdr));
  H->off_subs = int64_t(off);
  off += align16(sizeof(EstSub) * P->subs.size());
  H->off_ops = int64_t(off);
  off += align16(sizeof(EstOp) * P->ops.size());
  H->off_in = int64_t(off);
  off += align16(sizeof(EstIn) * P->ins.size());
  H->off_items = int64_t(off);
  off += align16(sizeof(EstItem) * P->items.size());
  H->off_tri = int64_t(off);
  off += align16(sizeof(TriSub) * P->tris.size());
  H->total_bytes = int64_t(off);
  H->max_suf = P->max_suf;
  H->max_rank = P->max_rank;
  const int64_t W1 = int64_t(w) + 1;
  H->scratch_per_cta = int64_t(align16(sizeof(i128) * size_t(int64_t(P->max_slots) * w + int64_t(P->max_suf) * W1 +
                                                             int64_t(P->max_in) * W1) +
                                       sizeof(int32_t) * size_t(int64_t(P->max_rank) * w)));
  H->ws_bytes = int64_t(est_ws_bytes(*H, H->grid, H->n_tri * d));
  return CMP_OK;
}

}  // namespace

extern "C" {

// Rows sorted per pass by the large-w path (bounds its workspace).
constexpr int64_t kPresortRowsPerPass = 64;

size_t cmp_presort_ws_bytes(int64_t n_rows, int32_t w) {
  if (n_rows <= 0 || w <= kPresortSmemMaxW || w > CMP_MAX_W) return 0;
  const int64_t rows = n_rows < kPresortRowsPerPass ? n_rows : kPresortRowsPerPass;
  return size_t(2 * rows * presort_padded(w) * int64_t(sizeof(unsigned long long)));
}

cmp_status cmp_cross_ranks(const uint32_t* abs_sorted_dev, const int32_t* perm_dev, int32_t k, int32_t d, int32_t w,
                           const int32_t* edge_id_host, int32_t* ranks_dev, void* stream) {
  // d only counts rows here (several tables' rows may be passed as one block when k = 1)
  if (k < 0 || k > CMP_MAX_SKETCHES || d < 1 || w < 1 || w > CMP_MAX_W) return CMP_EINVAL;
  if (int64_t(k) * k * d >= (int64_t(1) << 31)) return CMP_EINVAL;
  if (k > 0 && (!abs_sorted_dev || !perm_dev || !edge_id_host || !ranks_dev)) return CMP_EINVAL;
  return launch_cross_ranks(abs_sorted_dev, perm_dev, k, d, w, edge_id_host, ranks_dev,
                            reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

cmp_status cmp_cross_ranks_multi(const uint32_t* abs_sorted_dev, const int32_t* perm_dev, int32_t n_tables,
                                 const int32_t* k_host, const int32_t* edge_ids_host, int32_t d, int32_t w,
                                 int32_t* ranks_dev, void* stream) {
  if (n_tables < 0 || d < 1 || w < 1 || w > CMP_MAX_W || (n_tables > 0 && !k_host)) return CMP_EINVAL;
  int64_t blocks = 0, nk = 0;
  for (int32_t t = 0; t < n_tables; t++) {
    if (k_host[t] < 0 || k_host[t] > CMP_MAX_SKETCHES) return CMP_EINVAL;
    blocks += int64_t(k_host[t]) * k_host[t] * d;
    nk += k_host[t];
  }
  if (blocks >= (int64_t(1) << 31)) return CMP_EINVAL;
  if (nk > 0 && (!abs_sorted_dev || !perm_dev || !edge_ids_host || !ranks_dev)) return CMP_EINVAL;
  return launch_cross_ranks_multi(abs_sorted_dev, perm_dev, n_tables, k_host, edge_ids_host, d, w, ranks_dev,
                                  reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

cmp_status cmp_presort(const int32_t* counters_dev, int64_t n_rows, int32_t w, uint32_t* abs_sorted_dev,
                       int32_t* perm_dev, void* ws_dev, size_t ws_bytes, void* stream) {
  if (n_rows < 0 || w < 1 || w > CMP_MAX_W) return CMP_EINVAL;
  if (n_rows > 0 && (!counters_dev || !abs_sorted_dev || !perm_dev)) return CMP_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (w <= kPresortSmemMaxW)
    return launch_presort(counters_dev, n_rows, w, abs_sorted_dev, perm_dev, st) == cudaSuccess ? CMP_OK : CMP_ECUDA;
  if (n_rows == 0) return CMP_OK;
  if (!ws_dev || ws_bytes < cmp_presort_ws_bytes(n_rows, w)) return CMP_EWORKSPACE;
  const int64_t rows = n_rows < kPresortRowsPerPass ? n_rows : kPresortRowsPerPass;
  return launch_presort_large(counters_dev, n_rows, w, abs_sorted_dev, perm_dev, ws_dev, rows, st) == cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

cmp_status cmp_estimate_plan_bytes(const cmp_graph* graphs, int32_t n_graphs, int32_t d, int32_t w, int32_t n_sub,
                                   const int32_t* sub_graph, const uint64_t* sub_mask, const cmp_estimate_cfg* cfg,
                                   size_t* plan_bytes, size_t* ws_bytes) {
  if (!plan_bytes || !ws_bytes) return CMP_EINVAL;
  PlanOut P;
  EstPlanHdr H;
  const cmp_status st = plan_all(graphs, n_graphs, d, w, n_sub, sub_graph, sub_mask, cfg, &P, &H);
  if (st != CMP_OK) return st;
  *plan_bytes = size_t(H.total_bytes);
  *ws_bytes = size_t(H.ws_bytes);
  return CMP_OK;
}

cmp_status cmp_estimate_plan_encode(const cmp_graph* graphs, int32_t n_graphs, int32_t d, int32_t w, int32_t n_sub,
                                    const int32_t* sub_graph, const uint64_t* sub_mask, const cmp_estimate_cfg* cfg,
                                    void* plan_host, size_t plan_bytes) {
  if (!plan_host) return CMP_EINVAL;
  PlanOut P;
  EstPlanHdr H;
  const cmp_status st = plan_all(graphs, n_graphs, d, w, n_sub, sub_graph, sub_mask, cfg, &P, &H);
  if (st != CMP_OK) return st;
  if (plan_bytes < size_t(H.total_bytes)) return CMP_EWORKSPACE;
  unsigned char* b = static_cast<unsigned char*>(plan_host);
  std::memset(b, 0, size_t(H.total_bytes));
  std::memcpy(b, &H, sizeof(H));
  if (!P.subs.empty()) std::memcpy(b + H.off_subs, P.subs.data(), sizeof(EstSub) * P.subs.size());
  if (!P.ops.empty()) std::memcpy(b + H.off_ops, P.ops.data(), sizeof(EstOp) * P.ops.size());
  if (!P.ins.empty()) std::memcpy(b + H.off_in, P.ins.data(), sizeof(EstIn) * P.ins.size());
  if (!P.items.empty()) std::memcpy(b + H.off_items, P.items.data(), sizeof(EstItem) * P.items.size());
  if (!P.tris.empty()) std::memcpy(b + H.off_tri, P.tris.data(), sizeof(TriSub) * P.tris.size());
  return CMP_OK;
}

cmp_status cmp_estimate(const void* plan_host, const void* plan_dev, void* ws_dev, size_t ws_bytes, double* est_dev,
                        int64_t* row_est_dev, int32_t* status_dev, void* stream) {
  if (!plan_host || !plan_dev) return CMP_EINVAL;
  EstPlanHdr H;
  std::memcpy(&H, plan_host, sizeof(H));
  if (H.magic != kEstPlanMagic || H.version != kEstPlanVersion) return CMP_EINVAL;
  if (H.n_sub > 0 && !est_dev) return CMP_EINVAL;
  if (ws_bytes < size_t(H.ws_bytes) || (H.ws_bytes > 0 && !ws_dev)) return CMP_EWORKSPACE;
  const EstArgs a = est_args(H, static_cast<const unsigned char*>(plan_dev), static_cast<unsigned char*>(ws_dev),
                             H.grid, H.n_tri * H.d, status_dev);
  return launch_estimate(a, est_dev, row_est_dev, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? CMP_OK
                                                                                                          : CMP_ECUDA;
}

}  // extern "C"
