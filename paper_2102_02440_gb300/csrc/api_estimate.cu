// C ABI: presort and the batched sub-plan estimate (host planning + launches).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <utility>
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
  if (s->flags & ~int32_t(CMP_EST_GENERIC_ONLY | CMP_EST_CACHE_MESSAGES | CMP_EST_STAR_LATTICE | CMP_EST_NO_WIDE))
    return CMP_EINVAL;
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
  std::vector<StarFam> stars;
  std::vector<StarUnit> star_suf_units, star_lat_units;
  int64_t star_suf_words = 0, star_t_entries = 0, n_star_sub = 0;
  std::vector<int32_t> star_q;  // per family (StarFam.q_off): leaf set -> sub-plan, -1: none
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

// ---------------------------------------------------------------- cached subtree messages
// With CMP_EST_CACHE_MESSAGES, every tree sub-plan is rooted at its lowest table id and
// each non-leaf child subtree T, hanging from the root side by edge e, sends the message of
// T over e (the merged sketches of T contracted with each other and with T's sketch on e,
// Sec. 4.2 iterated).  The message depends on (graph, e, T) only, so one computed for a
// smaller subtree extends to every larger sub-plan that contains it (Sec. 4.2: (n+1)-D from
// n-D; Sec. 5: merged sketches cached).  A subtree message referenced by two or more
// parents (sub-plans or larger subtrees) is computed once, as a job, and cached; one with a
// single parent stays inline in that parent's operations.
struct JobNode {
  int32_t g, edge, root;
  uint64_t mask;
  int32_t refs, cid, level;
  std::vector<int32_t> kids;  // child subtree nodes (non-leaf children of root)
};
struct JobKeyHash {
  size_t operator()(const std::pair<uint64_t, uint64_t>& k) const {
    uint64_t h = k.first * 0x9E3779B97F4A7C15ull ^ (k.second + 0x632BE59BD9B4E019ull + (k.first << 6));
    h ^= h >> 29;
    return size_t(h * 0xBF58476D1CE4E5B9ull);
  }
};
struct CacheCtx {
  std::unordered_map<std::pair<uint64_t, uint64_t>, int32_t, JobKeyHash> key;  // (graph<<32 | edge, mask)
  std::vector<JobNode> nodes;
  int32_t lookup(int32_t gi, int32_t e, uint64_t m) const {
    const auto it = key.find({(uint64_t(uint32_t(gi)) << 32) | uint32_t(e), m});
    return it == key.end() ? -1 : it->second;
  }
};

inline bool touches(const cmp_graph& g, int e, int t) { return g.edge_u[e] == t || g.edge_v[e] == t; }
inline int other_end(const cmp_graph& g, int e, int t) { return g.edge_u[e] == t ? g.edge_v[e] : g.edge_u[e]; }

// Tables reachable from `start` inside `mask` without passing through `banned`.
uint64_t component(const cmp_graph& g, uint64_t mask, int start, int banned) {
  uint64_t seen = uint64_t(1) << start;
  int stack[CMP_MAX_TABLES], top = 0;
  stack[top++] = start;
  while (top) {
    const int t = stack[--top];
    for (int e = 0; e < g.n_edges; e++) {
      if (!touches(g, e, t)) continue;
      const int o = other_end(g, e, t);
      if (o == banned || !((mask >> o) & 1) || ((seen >> o) & 1)) continue;
      seen |= uint64_t(1) << o;
      stack[top++] = o;
    }
  }
  return seen;
}

// The node of subtree `m` sending over edge `e` (one end in m), created with its child
// nodes on first use.
int32_t job_node(const cmp_graph& g, int32_t gi, int32_t e, uint64_t m, CacheCtx* C) {
  const std::pair<uint64_t, uint64_t> k{(uint64_t(uint32_t(gi)) << 32) | uint32_t(e), m};
  const auto it = C->key.find(k);
  if (it != C->key.end()) return it->second;
  const int32_t id = int32_t(C->nodes.size());
  C->key.emplace(k, id);
  JobNode n;
  n.g = gi;
  n.edge = e;
  n.root = ((m >> g.edge_u[e]) & 1) ? g.edge_u[e] : g.edge_v[e];
  n.mask = m;
  n.refs = 0;
  n.cid = -1;
  n.level = -1;
  C->nodes.push_back(n);
  const int r = C->nodes[id].root;
  for (int e2 = 0; e2 < g.n_edges; e2++) {
    if (e2 == e || !touches(g, e2, r)) continue;
    const int o = other_end(g, e2, r);
    if (!((m >> o) & 1)) continue;
    const uint64_t sub = component(g, m, o, r);
    if (__builtin_popcountll(sub) < 2) continue;  // a leaf: its sketch is the message
    const int32_t kid = job_node(g, gi, e2, sub, C);
    C->nodes[kid].refs++;
    C->nodes[id].kids.push_back(kid);
  }
  return id;
}

// Registers the child subtrees of a tree sub-plan (rooted at its lowest table id); other
// sub-plans (single tables, cycles, invalid masks) register nothing.
void analyze_sub(const cmp_graph& g, int32_t gi, uint64_t mask, CacheCtx* C) {
  const int nt = g.n_tables;
  if (mask == 0 || (nt < 64 && (mask >> nt) != 0) || __builtin_popcountll(mask) < 2) return;
  int n_e = 0;
  for (int e = 0; e < g.n_edges; e++)
    if (((mask >> g.edge_u[e]) & 1) && ((mask >> g.edge_v[e]) & 1)) n_e++;
  int root = 0;
  while (!((mask >> root) & 1)) root++;
  if (component(g, mask, root, -1) != mask || n_e != __builtin_popcountll(mask) - 1) return;
  for (int e = 0; e < g.n_edges; e++) {
    if (!touches(g, e, root)) continue;
    const int o = other_end(g, e, root);
    if (!((mask >> o) & 1)) continue;
    const uint64_t sub = component(g, mask, o, root);
    if (__builtin_popcountll(sub) >= 2) C->nodes[job_node(g, gi, e, sub, C)].refs++;
  }
}

// Launch level of a cached node: 0 if it reads no cached message, else one more than the
// deepest cached message it reads (through its inline children).
int32_t job_level(int32_t id, CacheCtx* C) {
  JobNode& n = C->nodes[id];
  if (n.level >= 0) return n.level;
  int32_t lv = 0;
  std::vector<int32_t> st(n.kids.begin(), n.kids.end());
  while (!st.empty()) {
    const int32_t k = st.back();
    st.pop_back();
    if (C->nodes[k].cid >= 0) lv = std::max(lv, job_level(k, C) + 1);
    else st.insert(st.end(), C->nodes[k].kids.begin(), C->nodes[k].kids.end());
  }
  C->nodes[id].level = lv;
  return lv;
}

// Post-order operations of a spanning tree (BFS order `order` from `root`, tree edges
// marked), non-tree edges conditioned.  out_edge >= 0: the root sends over out_edge (whose
// other end is outside the tree) into the job's cached message.  With C, children whose
// subtree message is cached are read from the cache and their subtrees emit nothing.
cmp_status emit_ops(const cmp_graph& g, int32_t gi, const std::vector<int>& es, const std::vector<int>& order,
                    std::vector<int> parent_edge, const std::vector<char>& tree, int root, int out_edge,
                    const CacheCtx* C, PlanOut* P, EstSub* sb) {
  const int nt = g.n_tables;
  std::vector<int> ez = es;
  if (out_edge >= 0) {
    ez.insert(std::lower_bound(ez.begin(), ez.end(), out_edge), out_edge);
    parent_edge[root] = out_edge;
  }
  std::vector<int> deg(nt, 0);
  for (int e : es) deg[g.edge_u[e]]++, deg[g.edge_v[e]]++;
  auto is_leaf = [&](int t) { return t != root && deg[t] == 1; };
  auto end_of = [&](int e, int t) { return g.edge_u[e] == t ? 0 : 1; };
  // cached[t]: t's subtree message over its parent edge comes from the cache;
  // hidden[t]: t lies inside such a subtree
  std::vector<int> cached(nt, -1);
  std::vector<char> hidden(nt, 0);
  if (C) {
    std::vector<uint64_t> sub(nt, 0);
    for (size_t h = order.size(); h-- > 0;) {
      const int t = order[h];
      sub[t] |= uint64_t(1) << t;
      if (t != root) sub[other_end(g, parent_edge[t], t)] |= sub[t];
    }
    for (size_t h = 1; h < order.size(); h++) {
      const int t = order[h], p = other_end(g, parent_edge[t], t);
      hidden[t] = hidden[p] || (p != root && cached[p] >= 0);
      if (!hidden[t] && !is_leaf(t)) {
        const int32_t id = C->lookup(gi, parent_edge[t], sub[t]);
        if (id >= 0) cached[t] = C->nodes[id].cid;
      }
    }
  }
  sb->op_begin = int32_t(P->ops.size());
  std::vector<int> slot_of(nt, -1);
  std::vector<char> slot_busy;
  int32_t n_suf = 0;
  for (size_t h = order.size(); h-- > 0;) {
    const int t = order[h];
    if (is_leaf(t) || hidden[t] || (t != root && cached[t] >= 0)) continue;
    EstOp op;
    std::memset(&op, 0, sizeof(op));
    op.k = 0;
    op.p = -1;
    op.out_slot = -1;
    op.in_begin = int32_t(P->ins.size());
    std::vector<int> consumed;
    for (int e : ez) {
      if (!touches(g, e, t)) continue;
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
        const int child = other_end(g, e, t);
        if (is_leaf(child)) {
          x.kind = kInLeaf;
          x.msk = g.sketch[2 * e + end_of(e, child)];
        } else if (cached[child] >= 0) {
          x.kind = kInCache;
          x.slot = cached[child];
        } else {
          x.kind = kInSlot;
          x.slot = slot_of[child];
          consumed.push_back(slot_of[child]);
        }
      } else {
        x.kind = kInCond;
        x.slot = 0;  // ordinal among the conditioned edges (ascending edge id)
        for (int e2 : ez)
          if (e2 < e && !tree[e2]) x.slot++;
      }
      P->ins.push_back(x);
      op.k++;
    }
    if (op.p >= 0 && t != root) {  // output slot: a free slot not read by this operation
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
  sb->n_ops = int32_t(P->ops.size()) - sb->op_begin;
  if (sb->n_ops > kEstMaxOps || (sb->n_ops && int32_t(P->ins.size()) - P->ops[sb->op_begin].in_begin > kEstMaxSubIn))
    return CMP_EUNSUPPORTED;
  return CMP_OK;
}

// BFS spanning tree of `mask` from `root` over `es` (edges in id order).
void bfs_tree(const cmp_graph& g, const std::vector<int>& es, int root, std::vector<int>* order,
              std::vector<int>* parent_edge, std::vector<char>* tree) {
  const int nt = g.n_tables;
  order->assign(1, root);
  parent_edge->assign(nt, -1);
  tree->assign(g.n_edges, 0);
  std::vector<char> seen(nt, 0);
  seen[root] = 1;
  for (size_t h = 0; h < order->size(); h++) {
    const int t = (*order)[h];
    for (int e : es) {
      const int o = g.edge_u[e] == t ? g.edge_v[e] : (g.edge_v[e] == t ? g.edge_u[e] : -1);
      if (o < 0 || seen[o]) continue;
      seen[o] = 1;
      (*parent_edge)[o] = e;
      (*tree)[e] = 1;
      order->push_back(o);
    }
  }
}

std::vector<int> edges_within(const cmp_graph& g, uint64_t mask) {
  std::vector<int> es;
  for (int e = 0; e < g.n_edges; e++)
    if (((mask >> g.edge_u[e]) & 1) && ((mask >> g.edge_v[e]) & 1)) es.push_back(e);
  return es;
}

// Plan one sub-plan: spanning tree by BFS from the lowest table id (edges in id order),
// non-tree edges conditioned, post-order operations for every non-leaf table.
cmp_status plan_sub(const cmp_graph& g, int32_t gi, uint64_t mask, int32_t d, int32_t w, int32_t sub_index,
                    int32_t chunk, int32_t flags, const CacheCtx* C, int32_t star, uint32_t sbits, PlanOut* P) {
  const int nt = g.n_tables;
  if (mask == 0 || (nt < 64 && (mask >> nt) != 0)) return CMP_EINVAL;
  const std::vector<int> es = edges_within(g, mask);
  int root = 0;
  while (!((mask >> root) & 1)) root++;
  std::vector<int> order, parent_edge;
  std::vector<char> tree;
  bfs_tree(g, es, root, &order, &parent_edge, &tree);
  if (int(order.size()) != __builtin_popcountll(mask)) return CMP_EINVAL;  // not connected
  EstSub sb;
  std::memset(&sb, 0, sizeof(sb));
  sb.job = -1;
  sb.star = -1;
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
  if (star >= 0) {  // gathered from its family's lattice
    sb.star = star;
    sb.sbits = sbits;
    P->subs.push_back(sb);
    return CMP_OK;
  }
  std::vector<int> cond;
  for (int e : es)
    if (!tree[e]) cond.push_back(e);
  // every assignment of the conditioned edges' buckets: w^rho conditioning values (int32)
  if (cond.size() > size_t(kEstMaxCond)) return CMP_EUNSUPPORTED;
  int64_t n_cond_vals = 1;
  for (size_t k = 0; k < cond.size(); k++) n_cond_vals *= w;
  if (n_cond_vals > int64_t(INT32_MAX)) return CMP_EUNSUPPORTED;
  if (cond.size() == 1 && !(flags & CMP_EST_GENERIC_ONLY) && w <= kTriMaxW &&
      plan_triangle(g, es, tree, cond[0], mask, d, w, sub_index, P, &sb)) {
    P->subs.push_back(sb);
    return CMP_OK;
  }
  const cmp_status st = emit_ops(g, gi, es, order, parent_edge, tree, root, -1, cond.empty() ? C : nullptr, P, &sb);
  if (st != CMP_OK) return st;
  sb.cond = cond.empty() ? 0 : 1;
  const int32_t nv = int32_t(n_cond_vals);
  sb.n_chunks = cond.empty() ? 1 : int32_t((int64_t(nv) + chunk - 1) / chunk);
  // a wide tree whose only operation is a root with two or more inputs: its row is a sum over
  // the root's sorted positions, split into kRootSplit chunks (one CTA each)
  sb.split = cond.empty() && sb.n_ops == 1 && w >= kRootSplitMinW && P->ops[sb.op_begin].k >= 2 ? 1 : 0;
  if (sb.split) sb.n_chunks = kRootSplit;
  P->subs.push_back(sb);
  for (int i = 0; i < d; i++)
    for (int ch = 0; ch < sb.n_chunks; ch++) {
      EstItem it;
      it.sub = sub_index;
      it.row = i;
      if (sb.split) {
        it.c0 = int32_t(int64_t(w) * ch / kRootSplit);
        it.c1 = int32_t(int64_t(w) * (ch + 1) / kRootSplit);
      } else {
        it.c0 = cond.empty() ? 0 : int32_t(int64_t(ch) * chunk);
        it.c1 = cond.empty() ? 1 : int32_t(std::min<int64_t>(nv, int64_t(ch + 1) * chunk));
      }
      P->items.push_back(it);
    }
  return CMP_OK;
}

// The cached jobs, level by level: one EstSub each (after the n_sub sub-plans), its
// operations, and d items (one per sketch row) placed before every sub-plan item.
cmp_status plan_jobs(const cmp_graph* graphs, int32_t d, int32_t n_sub, CacheCtx* C, PlanOut* P, EstPlanHdr* H,
                     std::vector<EstItem>* job_items) {
  std::vector<int32_t> cached;  // node ids in cid order
  for (int32_t i = 0; i < int32_t(C->nodes.size()); i++)
    if (C->nodes[i].cid >= 0) cached.push_back(i);
  int32_t n_levels = 0;
  for (int32_t id : cached) n_levels = std::max(n_levels, job_level(id, C) + 1);
  if (n_levels > kEstMaxLevels) return CMP_EUNSUPPORTED;
  std::vector<EstSub> jsub(cached.size());
  for (int32_t lv = 0; lv < n_levels; lv++) {
    for (int32_t id : cached) {
      const JobNode& n = C->nodes[id];
      if (n.level != lv) continue;
      const cmp_graph& g = graphs[n.g];
      const std::vector<int> es = edges_within(g, n.mask);
      std::vector<int> order, parent_edge;
      std::vector<char> tree;
      bfs_tree(g, es, n.root, &order, &parent_edge, &tree);
      EstSub sb;
      std::memset(&sb, 0, sizeof(sb));
      sb.job = n.cid;
      sb.scale = 1.0;
      sb.tri = -1;
      sb.n_chunks = 1;
      sb.item_begin = int64_t(job_items->size());
      const cmp_status st = emit_ops(g, n.g, es, order, parent_edge, tree, n.root, n.edge, C, P, &sb);
      if (st != CMP_OK) return st;
      jsub[n.cid] = sb;
      for (int i = 0; i < d; i++) {
        EstItem it;
        it.sub = n_sub + n.cid;
        it.row = i;
        it.c0 = 0;
        it.c1 = 1;
        job_items->push_back(it);
      }
    }
    H->lvl_end[lv] = int64_t(job_items->size());
  }
  P->subs.insert(P->subs.end(), jsub.begin(), jsub.end());
  H->n_jobs = int64_t(cached.size());
  H->n_job_items = int64_t(job_items->size());
  H->n_levels = n_levels;
  return CMP_OK;
}

// Star families (CMP_EST_STAR_LATTICE): sub-plans whose edges all touch their lowest table
// (the root) and reach every other table once, grouped by (graph, root).  A family with
// leaf edges U (ascending id, K = |U| >= 3) is planned on the lattice when
// K 2^(K-1) <= 2 sum_S |S|^2 over its stars: the lattice's multiply-adds per sorted position
// against the generic contraction's products.  Its stars get star_of/sbits_of; the others
// stay on the generic path.
void plan_stars(const cmp_graph* graphs, int32_t n_sub, const int32_t* sub_graph, const uint64_t* sub_mask,
                int32_t d, int32_t w, PlanOut* P, std::vector<int32_t>* star_of, std::vector<uint32_t>* sbits_of) {
  struct Fam {
    int32_t g, root;
    std::vector<int32_t> qs;
    std::vector<std::vector<int>> edges;
  };
  std::vector<Fam> fams;
  std::unordered_map<uint64_t, int32_t> key;
  for (int32_t q = 0; q < n_sub; q++) {
    const cmp_graph& g = graphs[sub_graph[q]];
    const uint64_t mask = sub_mask[q];
    const int nt = g.n_tables;
    if (mask == 0 || (nt < 64 && (mask >> nt) != 0) || __builtin_popcountll(mask) < 2) continue;
    int root = 0;
    while (!((mask >> root) & 1)) root++;
    const std::vector<int> es = edges_within(g, mask);
    if (int(es.size()) != __builtin_popcountll(mask) - 1) continue;
    uint64_t reached = uint64_t(1) << root;
    bool star = true;
    for (int e : es) {
      if (!touches(g, e, root)) {
        star = false;
        break;
      }
      reached |= uint64_t(1) << other_end(g, e, root);
    }
    if (!star || reached != mask) continue;
    const uint64_t k = (uint64_t(uint32_t(sub_graph[q])) << 32) | uint32_t(root);
    auto it = key.find(k);
    int32_t f;
    if (it == key.end()) {
      f = int32_t(fams.size());
      key.emplace(k, f);
      fams.push_back(Fam{sub_graph[q], root, {}, {}});
    } else {
      f = it->second;
    }
    fams[f].qs.push_back(q);
    fams[f].edges.push_back(es);
  }
  for (const Fam& fm : fams) {
    std::vector<int> U;
    double sumsq = 0;
    for (const std::vector<int>& es : fm.edges) {
      U.insert(U.end(), es.begin(), es.end());
      sumsq += double(es.size()) * double(es.size());
    }
    std::sort(U.begin(), U.end());
    U.erase(std::unique(U.begin(), U.end()), U.end());
    const int K = int(U.size());
    if (K < 3 || K > CMP_MAX_SKETCHES || double(K) * double(int64_t(1) << (K - 1)) > 2.0 * sumsq) continue;
    const cmp_graph& g = graphs[fm.g];
    const int32_t fi = int32_t(P->stars.size());
    StarFam F;
    std::memset(&F, 0, sizeof(F));
    F.in_begin = int32_t(P->ins.size());
    F.K = K;
    const int k = K - 1;
    F.k2 = std::min(k, kStarMaxK2);
    F.k1 = k - F.k2;
    F.m1 = std::min(F.k1, std::max(0, 12 - F.k2));  // at most 2^12 entries per unit
    F.suf_off = P->star_suf_words;
    F.t_off = P->star_t_entries;
    F.q_off = int64_t(P->star_q.size());
    P->star_q.resize(P->star_q.size() + (size_t(1) << K), -1);
    P->star_suf_words += int64_t(d) * K * (int64_t(w) + 1);
    P->star_t_entries += int64_t(d) * K * (int64_t(1) << k);
    for (int e : U) {
      const int me = g.edge_u[e] == fm.root ? 0 : 1;
      EstIn x;
      std::memset(&x, 0, sizeof(x));
      x.s = g.sketch[2 * e + me];
      x.abs = g.abs_sorted[2 * e + me];
      x.perm = g.perm[2 * e + me];
      x.rk = g.ranks[2 * e + me];
      x.tslot = g.slot[2 * e + me];
      x.msk = g.sketch[2 * e + (1 - me)];
      x.kind = kInLeaf;
      x.slot = x.suf = -1;
      P->ins.push_back(x);
    }
    P->stars.push_back(F);
    for (int i = 0; i < d; i++)
      for (int b = 0; b < K; b++) P->star_suf_units.push_back(StarUnit{fi, i, b, -1});
    const int32_t n_blk = int32_t(1) << (F.k1 - F.m1);
    for (int i = 0; i < d; i++)
      for (int a = 0; a < K; a++)
        for (int32_t blk = 0; blk < n_blk; blk++) P->star_lat_units.push_back(StarUnit{fi, i, a, blk});
    for (size_t j = 0; j < fm.qs.size(); j++) {
      uint32_t bits = 0;
      for (int e : fm.edges[j]) bits |= 1u << int(std::lower_bound(U.begin(), U.end(), e) - U.begin());
      (*star_of)[fm.qs[j]] = fi;
      (*sbits_of)[fm.qs[j]] = bits;
      int32_t& slot = P->star_q[size_t(F.q_off) + bits];
      if (slot < 0) slot = fm.qs[j];  // a repeated leaf set keeps the first (the others: generic tier)
      P->n_star_sub++;
    }
  }
}

cmp_status plan_all(const cmp_graph* graphs, int32_t n_graphs, int32_t d, int32_t w, int32_t n_sub,
                    const int32_t* sub_graph, const uint64_t* sub_mask, const cmp_estimate_cfg* cfg, PlanOut* P,
                    EstPlanHdr* H, PlanOut* F) {
  if (!graphs || n_graphs < 1 || d < 1 || d > CMP_MAX_D || w < 1 || w > CMP_MAX_W || n_sub < 0) return CMP_EINVAL;
  EstShape shape;
  if (est_shape(cfg, &shape) != CMP_OK) return CMP_EINVAL;
  if (n_sub && (!sub_graph || !sub_mask)) return CMP_EINVAL;
  for (int32_t gi = 0; gi < n_graphs; gi++)
    if (!graph_ok(graphs[gi])) return CMP_EINVAL;
  for (int32_t q = 0; q < n_sub; q++)
    if (sub_graph[q] < 0 || sub_graph[q] >= n_graphs) return CMP_EINVAL;
  std::memset(H, 0, sizeof(*H));
  std::vector<int32_t> star_of(size_t(n_sub), -1);
  std::vector<uint32_t> sbits_of(size_t(n_sub), 0);
  if (shape.flags & CMP_EST_STAR_LATTICE) plan_stars(graphs, n_sub, sub_graph, sub_mask, d, w, P, &star_of, &sbits_of);
  CacheCtx cache;
  const bool use_cache = (shape.flags & CMP_EST_CACHE_MESSAGES) != 0;
  if (use_cache) {
    for (int32_t q = 0; q < n_sub; q++) analyze_sub(graphs[sub_graph[q]], sub_graph[q], sub_mask[q], &cache);
    for (int32_t i = 0, c = 0; i < int32_t(cache.nodes.size()); i++)  // referenced twice or more: cached
      if (cache.nodes[i].refs >= 2) cache.nodes[i].cid = c++;
  }
  for (int32_t q = 0; q < n_sub; q++) {
    const cmp_status st = plan_sub(graphs[sub_graph[q]], sub_graph[q], sub_mask[q], d, w, q, shape.cond_chunk,
                                   shape.flags, use_cache ? &cache : nullptr, star_of[q], sbits_of[q], P);
    if (st != CMP_OK) return st;
  }
  // items: cached jobs by level, then the sub-plans' generic items, then the triangle items
  std::vector<EstItem> job_items;
  if (use_cache) {
    const cmp_status st = plan_jobs(graphs, d, n_sub, &cache, P, H, &job_items);
    if (st != CMP_OK) return st;
  }
  const int64_t n_job = int64_t(job_items.size());
  const int64_t n_gen = n_job + int64_t(P->items.size());
  for (int32_t q = 0; q < n_sub; q++) P->subs[q].item_begin += P->subs[q].tri >= 0 ? n_gen : n_job;
  P->items.insert(P->items.begin(), job_items.begin(), job_items.end());
  P->items.insert(P->items.end(), P->tri_items.begin(), P->tri_items.end());
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
  H->n_star = int64_t(P->stars.size());
  H->off_star = int64_t(off);
  off += align16(sizeof(StarFam) * P->stars.size());
  H->n_star_suf_units = int64_t(P->star_suf_units.size());
  H->n_star_units = H->n_star_suf_units + int64_t(P->star_lat_units.size());
  H->off_star_units = int64_t(off);
  off += align16(sizeof(StarUnit) * size_t(H->n_star_units));
  H->star_suf_words = P->star_suf_words;
  H->star_t_entries = P->star_t_entries;
  H->off_star_q = int64_t(off);
  H->n_star_q = int64_t(P->star_q.size());
  off += align16(sizeof(int32_t) * P->star_q.size());
  // exact tier beyond int128: the sub-plans on the generic path alone (the main arrays when
  // they already are), evaluated again modulo the primes for the rows found out of range
  H->wide = (shape.flags & CMP_EST_NO_WIDE) ? 0 : 1;
  F->subs.clear();
  if (H->wide) {
    const bool own = !P->stars.empty() || !P->tris.empty() || n_job > 0;
    if (own) {
      for (int32_t q = 0; q < n_sub; q++) {
        const cmp_status st = plan_sub(graphs[sub_graph[q]], sub_graph[q], sub_mask[q], d, w, q, shape.cond_chunk,
                                       CMP_EST_GENERIC_ONLY, nullptr, -1, 0, F);
        if (st != CMP_OK) return st;
      }
      H->wide_off_subs = int64_t(off);
      off += align16(sizeof(EstSub) * F->subs.size());
      H->wide_off_ops = int64_t(off);
      off += align16(sizeof(EstOp) * F->ops.size());
      H->wide_off_in = int64_t(off);
      off += align16(sizeof(EstIn) * F->ins.size());
      H->wide_off_items = int64_t(off);
      off += align16(sizeof(EstItem) * F->items.size());
      H->wide_n_items = int64_t(F->items.size());
    } else {
      H->wide_off_subs = H->off_subs;
      H->wide_off_ops = H->off_ops;
      H->wide_off_in = H->off_in;
      H->wide_off_items = H->off_items;
      H->wide_n_items = n_gen;
    }
    const PlanOut& G = own ? *F : *P;
    int64_t units = 0;  // every row of every sub-plan, once per conditioning chunk
    for (const EstSub& sb : G.subs) units += int64_t(d) * std::max<int32_t>(1, sb.n_chunks);
    H->wide_unit_cap = int32_t(std::min<int64_t>(std::max<int64_t>(units, 1), kWideUnitMax));
    H->wide_max_slots = G.max_slots;
    H->wide_max_in = G.max_in;
    H->wide_max_suf = G.max_suf;
    H->wide_qcap = int32_t(std::min<int64_t>(int64_t(n_sub) * d, kWideQueueMax));
    H->wide_scratch_per_cta = int64_t(align16(
        sizeof(uint64_t) * size_t(int64_t(G.max_slots) * w + int64_t(G.max_suf) * (int64_t(w) + 1) +
                                  int64_t(std::max(G.max_in, 1)) * (int64_t(w) + 1))));
    // its own grid: kWideCtasPerSm CTAs per SM, as many as fit in kWideScratchBudget, and no
    // more than its (unit, prime) jobs (at least one)
    H->wide_grid = int32_t(std::max<int64_t>(
        1, std::min<int64_t>({int64_t(sm_count()) * kWideCtasPerSm,
                              kWideScratchBudget / std::max<int64_t>(H->wide_scratch_per_cta, 1),
                              int64_t(H->wide_unit_cap) * kWideMods})));
  }
  H->total_bytes = int64_t(off);
  H->max_suf = P->max_suf;
  H->max_rank = P->max_rank;
  const int64_t W1 = int64_t(w) + 1;
  H->scratch_per_cta = int64_t(align16(sizeof(i128) * size_t(int64_t(P->max_slots) * w + int64_t(P->max_suf) * W1 +
                                                             int64_t(P->max_in) * W1) +
                                       sizeof(int32_t) * size_t(int64_t(P->max_rank) * w)));
  H->ws_bytes = int64_t(est_ws_bytes(*H, H->grid, H->n_tri * d, H->wide_grid));
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
  PlanOut P, F;
  EstPlanHdr H;
  const cmp_status st = plan_all(graphs, n_graphs, d, w, n_sub, sub_graph, sub_mask, cfg, &P, &H, &F);
  if (st != CMP_OK) return st;
  *plan_bytes = size_t(H.total_bytes);
  *ws_bytes = size_t(H.ws_bytes);
  return CMP_OK;
}

cmp_status cmp_estimate_plan_encode(const cmp_graph* graphs, int32_t n_graphs, int32_t d, int32_t w, int32_t n_sub,
                                    const int32_t* sub_graph, const uint64_t* sub_mask, const cmp_estimate_cfg* cfg,
                                    void* plan_host, size_t plan_bytes) {
  if (!plan_host) return CMP_EINVAL;
  PlanOut P, F;
  EstPlanHdr H;
  const cmp_status st = plan_all(graphs, n_graphs, d, w, n_sub, sub_graph, sub_mask, cfg, &P, &H, &F);
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
  if (!P.stars.empty()) std::memcpy(b + H.off_star, P.stars.data(), sizeof(StarFam) * P.stars.size());
  if (!P.star_suf_units.empty())
    std::memcpy(b + H.off_star_units, P.star_suf_units.data(), sizeof(StarUnit) * P.star_suf_units.size());
  if (!P.star_lat_units.empty())
    std::memcpy(b + H.off_star_units + sizeof(StarUnit) * P.star_suf_units.size(), P.star_lat_units.data(),
                sizeof(StarUnit) * P.star_lat_units.size());
  if (!P.star_q.empty()) std::memcpy(b + H.off_star_q, P.star_q.data(), sizeof(int32_t) * P.star_q.size());
  if (!F.subs.empty()) {  // the exact tier's own generic plan
    std::memcpy(b + H.wide_off_subs, F.subs.data(), sizeof(EstSub) * F.subs.size());
    if (!F.ops.empty()) std::memcpy(b + H.wide_off_ops, F.ops.data(), sizeof(EstOp) * F.ops.size());
    if (!F.ins.empty()) std::memcpy(b + H.wide_off_in, F.ins.data(), sizeof(EstIn) * F.ins.size());
    if (!F.items.empty()) std::memcpy(b + H.wide_off_items, F.items.data(), sizeof(EstItem) * F.items.size());
  }
  return CMP_OK;
}

cmp_status cmp_estimate_plan_stats(const void* plan_host, cmp_estimate_plan_info* info) {
  if (!plan_host || !info) return CMP_EINVAL;
  EstPlanHdr H;
  std::memcpy(&H, plan_host, sizeof(H));
  if (H.magic != kEstPlanMagic || H.version != kEstPlanVersion) return CMP_EINVAL;
  info->n_sub = H.n_sub;
  info->n_items = H.n_items;
  info->n_ops = H.n_ops;
  info->n_jobs = H.n_jobs;
  info->n_job_items = H.n_job_items;
  info->n_tri = H.n_tri;
  info->n_levels = H.n_levels;
  info->grid = H.grid;
  info->n_star = H.n_star;
  info->n_star_sub = 0;
  info->n_star_entries = H.star_t_entries;
  const EstSub* subs = reinterpret_cast<const EstSub*>(static_cast<const unsigned char*>(plan_host) + H.off_subs);
  for (int64_t q = 0; q < H.n_sub; q++) info->n_star_sub += subs[q].star >= 0 ? 1 : 0;
  return CMP_OK;
}

cmp_status cmp_estimate(const void* plan_host, const void* plan_dev, void* ws_dev, size_t ws_bytes, double* est_dev,
                        int64_t* row_est_dev, int32_t* status_dev, void* stream) {
  return cmp_estimate_ex(plan_host, plan_dev, ws_dev, ws_bytes, est_dev, row_est_dev, nullptr, status_dev, stream);
}

cmp_status cmp_estimate_ex(const void* plan_host, const void* plan_dev, void* ws_dev, size_t ws_bytes, double* est_dev,
                           int64_t* row_est_dev, int64_t* wide_rows_dev, int32_t* status_dev, void* stream) {
  if (!plan_host || !plan_dev) return CMP_EINVAL;
  EstPlanHdr H;
  std::memcpy(&H, plan_host, sizeof(H));
  if (H.magic != kEstPlanMagic || H.version != kEstPlanVersion) return CMP_EINVAL;
  if (H.n_sub > 0 && !est_dev) return CMP_EINVAL;
  if (ws_bytes < size_t(H.ws_bytes) || (H.ws_bytes > 0 && !ws_dev)) return CMP_EWORKSPACE;
  const EstArgs a = est_args(H, static_cast<const unsigned char*>(plan_dev), static_cast<unsigned char*>(ws_dev),
                             H.grid, H.n_tri * H.d, status_dev, H.wide_grid);
  return launch_estimate(a, H, est_dev, row_est_dev, reinterpret_cast<cudaStream_t>(stream), wide_rows_dev) ==
                 cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

}  // extern "C"
