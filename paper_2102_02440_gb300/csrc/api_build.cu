// C ABI: general entry points, hash parameters, single-table and batched builds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace cmpk {

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 152;  // GB300; only used to size grids when no device is visible
  }
  return n;
}

size_t smem_optin_bytes() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 232448;
  }
  return size_t(n);
}

namespace {
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cmp_status check_table(const cmp_table* t, int32_t d, int32_t w, int32_t n_edges) {
  if (!t || d < 1 || d > CMP_MAX_D || w < 1 || w > CMP_MAX_W || n_edges < 0) return CMP_EINVAL;
  if (t->n_rows < 0 || t->n_rows > 2147483647LL) return CMP_EINVAL;
  if (t->n_cols < 0 || t->n_cols > CMP_MAX_COLS || t->n_preds < 0 || t->n_preds > CMP_MAX_PREDS ||
      t->n_sketches < 0 || t->n_sketches > CMP_MAX_SKETCHES)
    return CMP_EINVAL;
  if ((t->n_cols && !t->cols) || (t->n_preds && !t->preds) || (t->n_sketches && (!t->key_col || !t->edge_id)))
    return CMP_EINVAL;
  for (int c = 0; c < t->n_cols; c++) {
    if (t->cols[c].dtype != CMP_I32 && t->cols[c].dtype != CMP_I64) return CMP_EINVAL;
    if (t->n_rows > 0 && !t->cols[c].data) return CMP_EINVAL;
    if (t->cols[c].flags & ~(CMP_COL_UNIQUE | CMP_COL_DOMAIN)) return CMP_EINVAL;
    if ((t->cols[c].flags & CMP_COL_DOMAIN) && !(t->cols[c].dom_lo < t->cols[c].dom_hi)) return CMP_EINVAL;
  }
  for (int q = 0; q < t->n_preds; q++) {
    const cmp_pred& p = t->preds[q];
    if (p.col < 0 || p.col >= t->n_cols || p.op < CMP_RANGE || p.op > CMP_IN_BITMAP) return CMP_EINVAL;
    if (p.op == CMP_IN_BITMAP && (p.bitmap_nbits < 0 || (p.bitmap_nbits > 0 && !p.bitmap))) return CMP_EINVAL;
  }
  for (int s = 0; s < t->n_sketches; s++) {
    if (t->key_col[s] < 0 || t->key_col[s] >= t->n_cols) return CMP_EINVAL;
    if (t->edge_id[s] < 0 || t->edge_id[s] >= n_edges) return CMP_EINVAL;
  }
  if (!(t->sample_rate >= 0.0 && t->sample_rate <= 1.0)) return CMP_EINVAL;  // NaN fails too
  return CMP_OK;
}

DevTable to_dev(const cmp_table* t, int32_t* counters, int64_t* survivors) {
  DevTable D;
  std::memset(&D, 0, sizeof(D));
  D.n_rows = t->n_rows;
  D.n_cols = t->n_cols;
  D.n_preds = t->n_preds;
  D.n_sketches = t->n_sketches;
  D.vec_ok = 1;
  for (int c = 0; c < t->n_cols; c++) {
    D.col[c] = t->cols[c].data;
    D.dtype[c] = t->cols[c].dtype;
    if (!aligned16(t->cols[c].data)) D.vec_ok = 0;
  }
  for (int q = 0; q < t->n_preds; q++) {
    const cmp_pred& p = t->preds[q];
    D.pred[q].col = p.col;
    D.pred[q].op = p.op;
    D.pred[q].lo = p.lo;
    D.pred[q].hi = p.hi;
    D.pred[q].bitmap = p.bitmap;
    D.pred[q].nbits = p.op == CMP_IN_BITMAP ? p.bitmap_nbits : 0;
  }
  for (int s = 0; s < t->n_sketches; s++) {
    D.key_col[s] = t->key_col[s];
    D.edge_id[s] = t->edge_id[s];
  }
  D.sample_seed = t->sample_seed;
  D.sample_keep = sample_keep_of(t->sample_rate);
  D.filtered = (t->n_preds > 0 || D.sample_keep != 0) ? 1 : 0;
  D.counters = counters;
  D.survivors = survivors;
  for (int c = 0; c < CMP_MAX_COLS; c++) D.agg[c] = -1;
  return D;
}

namespace {

struct SplitMix64 {  // Steele, Lea & Flood 2014
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

uint32_t next_pow2(uint32_t v) {
  uint32_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Shape common to one launch (single or batched).  max_total_pairs = largest k*d.
cmp_status choose_shape(const cmp_build_cfg* cfg, int32_t d, int32_t w, int32_t max_total_pairs, BuildShape* out) {
  BuildShape s;
  std::memset(&s, 0, sizeof(s));
  const size_t optin = smem_optin_bytes();
  const size_t pair_bytes = size_t(w) * 4;
  int mode = (cfg && cfg->mode > 0) ? cfg->mode : 0;
  if (mode < 0 || mode > 2) return CMP_EINVAL;
  const int pairs_all = std::max(max_total_pairs, 1);
  // Shared-memory slabs pay off when one small slab holds every pair of the table (no
  // column re-reads, several CTAs per SM); otherwise L2-resident counters do better.
  if (mode == 0) mode = size_t(pairs_all) * pair_bytes <= 48 * 1024 ? 1 : 2;
  s.threads = (cfg && cfg->threads > 0) ? cfg->threads : (mode == 2 ? 1024 : 512);
  s.tile_rows = (cfg && cfg->tile_rows > 0) ? cfg->tile_rows : (mode == 2 ? 4096 : 2048);
  s.dedupe = (cfg && cfg->dedupe >= 0) ? (cfg->dedupe ? 1 : 0) : 1;
  if (s.threads < 32 || s.threads > 1024 || s.threads % 32) return CMP_EINVAL;
  if (s.tile_rows < 128 || s.tile_rows > 16384 || s.tile_rows % 128) return CMP_EINVAL;
  // the map holds up to 2 entries per tile row; aggregated items use it as 64 entries per warp
  s.map_slots = s.dedupe ? int32_t(next_pow2(uint32_t(std::max(2 * s.tile_rows, 2 * s.threads)))) : 0;
  if (s.dedupe && s.map_slots > 8 * s.threads) return CMP_EINVAL;  // compaction keeps <= 8 slots per thread
  // overhead of everything but the private counters, with the parameter area sized for all pairs
  BuildShape probe = s;
  probe.mode = 2;
  probe.max_pairs = pairs_all;
  const size_t overhead = build_smem_bytes(probe, w) + 1024;
  if (mode == 1 && pair_bytes + overhead > optin) return CMP_EINVAL;
  s.mode = mode;
  int ctas_per_sm = (cfg && cfg->ctas_per_sm > 0) ? cfg->ctas_per_sm : 0;
  if (mode == 1) {
    if (!ctas_per_sm) ctas_per_sm = pair_bytes * std::min(pairs_all, 11) > 64 * 1024 ? 1 : 2;
    const size_t per_cta = optin / size_t(ctas_per_sm) - (ctas_per_sm > 1 ? 1024 : 0);
    if (per_cta <= overhead) return CMP_EINVAL;
    int pps = int(std::min<size_t>(size_t(pairs_all), (per_cta - overhead) / pair_bytes));
    if (cfg && cfg->pairs_per_slab > 0) pps = std::min(cfg->pairs_per_slab, pairs_all);
    if (pps < 1) return CMP_EINVAL;
    const int n_slabs = (pairs_all + pps - 1) / pps;
    pps = (pairs_all + n_slabs - 1) / n_slabs;  // equal slabs
    s.pairs_per_slab = pps;
    s.smem_pairs = pps;
    s.max_pairs = pps;
  } else {
    if (!ctas_per_sm) ctas_per_sm = 2;
    s.pairs_per_slab = pairs_all;
    s.smem_pairs = 0;
    s.max_pairs = pairs_all;
  }
  s.ctas_per_slab = ctas_per_sm;  // temporarily: CTAs per SM
  s.smem_bytes = build_smem_bytes(s, w);
  if (s.smem_bytes > optin) return CMP_EINVAL;
  *out = s;
  return CMP_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace
}  // namespace cmpk

using namespace cmpk;

extern "C" {

int32_t cmp_abi_version(void) { return CMP_ABI_VERSION; }

const char* cmp_status_str(cmp_status s) {
  switch (s) {
    case CMP_OK: return "ok";
    case CMP_EINVAL: return "invalid argument";
    case CMP_EUNSUPPORTED: return "unsupported input";
    case CMP_EOVERFLOW: return "exact integer overflow";
    case CMP_ECUDA: return "CUDA error";
    case CMP_EWORKSPACE: return "workspace or plan buffer too small";
    case CMP_ETIMEOUT: return "bounded device wait ran out";
    default: return "unknown status";
  }
}

cmp_status cmp_hash_params(uint64_t seed, int32_t n_edges, int32_t d, cmp_hash* out_host) {
  if (n_edges < 0 || d < 1 || d > CMP_MAX_D || (n_edges > 0 && !out_host)) return CMP_EINVAL;
  SplitMix64 g{seed};
  for (int32_t e = 0; e < n_edges; e++)
    for (int32_t i = 0; i < d; i++) {
      uint64_t f[6];
      for (int k = 0; k < 6; k++) {
        const uint64_t v = g.next() >> 3;
        f[k] = v == kP61 ? 0 : v;
      }
      if (f[0] == 0) f[0] = 1;
      cmp_hash& h = out_host[size_t(e) * d + i];
      h.a = f[0], h.b = f[1], h.c0 = f[2], h.c1 = f[3], h.c2 = f[4], h.c3 = f[5];
    }
  return CMP_OK;
}

cmp_status cmp_sketch_build(const cmp_table* table, int32_t d, int32_t w, const cmp_hash* hash_dev, int32_t n_edges,
                            int32_t* counters_dev, int64_t* survivors_dev, int32_t* status_dev,
                            const cmp_build_cfg* cfg, void* stream) {
  cmp_status st = check_table(table, d, w, n_edges);
  if (st != CMP_OK) return st;
  if (!survivors_dev || (table->n_sketches && (!counters_dev || !hash_dev))) return CMP_EINVAL;
  const int32_t total_pairs = table->n_sketches * d;
  BuildShape s;
  st = choose_shape(cfg, d, w, total_pairs, &s);
  if (st != CMP_OK) return st;
  cudaStream_t cs = as_stream(stream);
  const size_t cbytes = size_t(total_pairs) * w * sizeof(int32_t);
  if (cbytes && cudaMemsetAsync(counters_dev, 0, cbytes, cs) != cudaSuccess) return CMP_ECUDA;
  if (cudaMemsetAsync(survivors_dev, 0, sizeof(int64_t), cs) != cudaSuccess) return CMP_ECUDA;
  if (table->n_rows == 0) return CMP_OK;
  const int n_slabs = total_pairs ? (total_pairs + s.pairs_per_slab - 1) / s.pairs_per_slab : 1;
  const int64_t n_tiles = (table->n_rows + s.tile_rows - 1) / s.tile_rows;
  const int target = sm_count() * s.ctas_per_slab;
  s.ctas_per_slab = int(std::max<int64_t>(1, std::min<int64_t>(n_tiles, (target + n_slabs - 1) / n_slabs)));
  s.grid = n_slabs * s.ctas_per_slab;
  BuildArgs a;
  std::memset(&a, 0, sizeof(a));
  a.table = to_dev(table, counters_dev, survivors_dev);
  a.hash = hash_dev;
  a.status = status_dev;
  a.d = d, a.w = w, a.n_edges = n_edges;
  a.threads = s.threads, a.tile_rows = s.tile_rows, a.map_slots = s.map_slots;
  a.max_pairs = s.max_pairs, a.smem_pairs = s.smem_pairs;
  a.pairs_per_slab = s.pairs_per_slab, a.ctas_per_slab = s.ctas_per_slab;
  return launch_build(a, s, cs) == cudaSuccess ? CMP_OK : CMP_ECUDA;
}

// ---------------------------------------------------------------- batched build plan
// blob: [BuildPlanHdr][DevTable x n_tables][BuildItem x n_items][int32 cta_item x grid]
//       [ZeroSpan x n_zero][AggCol x n_agg][CountItem x n_cnt_items]

// Key aggregation: tables with at least this many rows (auto mode), count arrays of at
// most this many slots (a column whose key range is wider keeps the per-row path).
constexpr int64_t kAggMinRows = int64_t(1) << 18;
constexpr int64_t kAggMaxCap = int64_t(1) << 27;

// Unique-key kernel: shared-memory budget of a slab's counters (room is left on the SM for
// a CTA of the counting pass), rows per tile.
constexpr size_t kUniqSmemBudget = size_t(128) << 10;
constexpr int32_t kUniqTileRows = 4096;
constexpr int32_t kUniqThreadsHost = 512;

// Presence bitmaps (dense kernel): a unique column with a declared domain in a table
// without predicates or sample, whose domain is at most kDenseMaxFill times its rows (the
// kernel steps through every key of the domain) and at most kDenseMaxSpan keys.
constexpr int64_t kDenseMaxFill = 4;
constexpr int64_t kDenseMaxSpan = int64_t(1) << 32;

struct BuildPlanParts {
  BuildShape shape;
  std::vector<UniqSlab> uslabs;
  std::vector<UniqItem> uitems;
  std::vector<int32_t> u_cta_item;  // [u_grid + 1]
  int32_t u_pack16 = 0, u_words = 0;
  std::vector<UniqSlab> dslabs;     // dense kernel
  std::vector<UniqItem> ditems;
  std::vector<int32_t> d_cta_item;  // [d_grid + 1]
  int32_t d_words = 0, n_presence = 0;
  std::vector<uint32_t> uniq_mask;  // [table]
  std::vector<int32_t> surv_by;     // [table]
  std::vector<BuildItem> items;
  std::vector<int32_t> cta_item;
  std::vector<AggCol> aggs;
  std::vector<CountItem> cnt_items;
  int64_t cnt_total_chunks = 0;
  int32_t cnt_grid = 0;
  int64_t cnt_split = 0;  // > 0: two launches, the tables with presence columns first
  int32_t d_cut = 1024;   // split pass: the dense kernel's share beside the second counting launch
  int32_t cnt_grid_b = 0;
  int64_t hash_total_chunks = 0;
  int32_t hash_max_pairs = 1, hash_grid = 0;
  std::vector<std::vector<int32_t>> col_agg;  // [table][col] AggCol index or -1
  size_t bytes = 0, ws_bytes = 0;
  int32_t cache_slots = 256, cache_cols = 0;  // counting pass
};

static uint64_t next_pow2_64(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

static cmp_status plan_layout(const cmp_table* tables, int32_t n_tables, int32_t d, int32_t w,
                              const cmp_build_cfg* cfg, int32_t n_edges_check, BuildPlanParts* P) {
  if (n_tables < 1 || !tables) return CMP_EINVAL;
  int32_t max_pairs = 1;
  for (int32_t t = 0; t < n_tables; t++) {
    cmp_status st = check_table(&tables[t], d, w, n_edges_check);
    if (st != CMP_OK) return st;
    max_pairs = std::max(max_pairs, tables[t].n_sketches * d);
  }
  BuildShape s;
  cmp_status st = choose_shape(cfg, d, w, max_pairs, &s);
  if (st != CMP_OK) return st;
  const int agg_mode = cfg ? cfg->aggregate : -1;
  if (agg_mode < -1 || agg_mode > 1) return CMP_EINVAL;
  if (agg_mode == 1 && !s.dedupe) return CMP_EINVAL;  // aggregated items use the tile map's entry lists
  const int ctas_per_sm = s.ctas_per_slab;
  const int R = s.tile_rows;
  // Key columns: declared unique -> unique-key kernel (when its slab fits in shared
  // memory); else aggregated (large tables); else the row kernel.
  const int uniq_mode = cfg ? cfg->unique : 0;
  if (uniq_mode < -1 || uniq_mode > 1) return CMP_EINVAL;
  P->u_pack16 = size_t(w) * 4 > kUniqSmemBudget ? 1 : 0;
  const bool uniq_fits = size_t(w) * (P->u_pack16 ? 2 : 4) <= kUniqSmemBudget;
  P->uniq_mask.assign(n_tables, 0u);
  P->surv_by.assign(n_tables, kSurvRow);
  P->col_agg.assign(n_tables, std::vector<int32_t>(CMP_MAX_COLS, -1));
  P->aggs.clear();
  size_t ws = al256(16 * size_t(n_tables) * CMP_MAX_SKETCHES + 32);  // stats + chunk counters (upper bound)
  for (int32_t t = 0; t < n_tables; t++) {
    const cmp_table& tb = tables[t];
    const bool agg_on = tb.n_sketches > 0 && tb.n_rows > 0 && s.dedupe &&
                        (agg_mode == 1 || (agg_mode == -1 && tb.n_rows >= kAggMinRows));
    const bool unfiltered = tb.n_preds == 0 && !(tb.sample_rate > 0.0 && tb.sample_rate < 1.0);
    for (int k = 0; k < tb.n_sketches; k++) {
      const int c = tb.key_col[k];
      const cmp_col& col = tb.cols[c];
      if (uniq_mode >= 0 && uniq_fits && (col.flags & CMP_COL_UNIQUE)) {
        const uint64_t span = (col.flags & CMP_COL_DOMAIN) ? uint64_t(col.dom_hi) - uint64_t(col.dom_lo) : 0;
        if (unfiltered && span > 0 && span <= uint64_t(kDenseMaxSpan) &&
            span <= uint64_t(kDenseMaxFill) * uint64_t(tb.n_rows)) {
          if (P->col_agg[t][c] >= 0) continue;
          AggCol a;  // presence bitmap over the declared domain
          std::memset(&a, 0, sizeof(a));
          a.table = t;
          a.col = c;
          a.cap = int64_t(span);
          a.base = col.dom_lo;
          a.mask = ~0ull;
          a.kind = kAggPresence;
          P->col_agg[t][c] = int32_t(P->aggs.size());
          P->aggs.push_back(a);
          continue;
        }
        P->uniq_mask[t] |= 1u << c;
        continue;
      }
      if (!agg_on || P->col_agg[t][c] >= 0) continue;
      AggCol a;
      std::memset(&a, 0, sizeof(a));
      a.table = t;
      a.col = c;
      const uint64_t dom = (col.flags & CMP_COL_DOMAIN) ? uint64_t(col.dom_hi) - uint64_t(col.dom_lo) : 0;
      if (dom > 0 && dom <= uint64_t(kAggMaxCap)) {  // the declared domain, slot = key - dom_lo
        a.cap = int64_t(dom);
        a.base = col.dom_lo;
        a.mask = ~0ull;
      } else {  // a power of two, slot = key mod cap
        a.cap = int64_t(next_pow2_64(uint64_t(std::min<int64_t>(tb.n_rows, kAggMaxCap))));
        a.base = 0;
        a.mask = uint64_t(a.cap) - 1;
      }
      P->col_agg[t][c] = int32_t(P->aggs.size());
      P->aggs.push_back(a);
    }
    bool has_agg = false;
    for (int c = 0; c < CMP_MAX_COLS; c++) has_agg |= P->col_agg[t][c] >= 0;
    P->surv_by[t] = has_agg ? kSurvCount : (P->uniq_mask[t] ? kSurvUniq : kSurvRow);
  }
  if (P->aggs.size() > size_t(n_tables) * CMP_MAX_SKETCHES) return CMP_EINVAL;
  for (AggCol& a : P->aggs) {
    a.off = int64_t(ws);
    // whole int4 words: the zeroing kernel writes them
    ws += a.kind == kAggPresence ? al256(sizeof(uint32_t) * size_t(presence_words(a.cap)) + sizeof(PresenceCheck))
                                 : al256(16 * size_t((a.cap + 3) / 4));
  }
  P->ws_bytes = P->aggs.empty() ? 0 : ws;
  // unique-key slabs and their items: each CTA gets about the same number of tiles; the
  // slabs of one column (same table, same tiles) get the same row split, so CTAs reading
  // the same rows run side by side
  P->uslabs.clear();
  P->uitems.clear();
  P->u_cta_item.assign(1, 0);
  P->u_words = 0;
  {
    struct Group {
      int32_t t, c, first, n;  // slabs [first, first + n)
      int64_t tiles;
    };
    std::vector<Group> groups;
    int64_t total_tiles = 0;
    for (int32_t t = 0; t < n_tables; t++) {
      const cmp_table& tb = tables[t];
      if (!P->uniq_mask[t] || tb.n_rows == 0) continue;
      const int64_t tiles = (tb.n_rows + kUniqTileRows - 1) / kUniqTileRows;
      for (int c = 0; c < tb.n_cols; c++) {
        if (!((P->uniq_mask[t] >> c) & 1u)) continue;
        std::vector<int32_t> pairs;
        for (int k = 0; k < tb.n_sketches; k++)
          if (tb.key_col[k] == c)
            for (int i = 0; i < d; i++) pairs.push_back(k * d + i);
        const int max_pps = P->u_pack16 ? 1
                                         : int(std::max<size_t>(1, std::min<size_t>(kUniqMaxPairs,
                                                                                    kUniqSmemBudget / (size_t(w) * 4))));
        const int n_sl = int((pairs.size() + max_pps - 1) / max_pps);
        const int pps = int((pairs.size() + n_sl - 1) / n_sl);
        Group g{t, c, int32_t(P->uslabs.size()), 0, tiles};
        for (size_t b = 0; b < pairs.size(); b += pps) {
          UniqSlab sl;
          std::memset(&sl, 0, sizeof(sl));
          sl.table = t;
          sl.col = c;
          sl.n_pairs = int32_t(std::min(pairs.size() - b, size_t(pps)));
          for (int q = 0; q < sl.n_pairs; q++) sl.pair[q] = pairs[b + q];
          P->u_words = std::max<int32_t>(P->u_words, P->u_pack16 ? int32_t((w + 1) / 2) : sl.n_pairs * w);
          P->uslabs.push_back(sl);
          g.n++;
        }
        total_tiles += tiles * g.n;
        groups.push_back(g);
      }
    }
    if (!groups.empty()) {
      const double avg = std::max(1.0, double(total_tiles) / double(sm_count()));
      std::vector<bool> counted(n_tables, false);
      auto add_item = [&](int32_t slab, int64_t rb, int64_t re) {
        UniqItem it;
        it.slab = slab;
        it.count_surv = 0;
        it.row_begin = rb;
        it.row_end = re;
        P->uitems.push_back(it);
      };
      for (const Group& g : groups) {
        const int64_t rows = tables[g.t].n_rows;
        const bool count_first = P->surv_by[g.t] == kSurvUniq && !counted[g.t];
        if (double(g.tiles) >= 0.5 * avg) {
          // every slab split into n equal row ranges, one CTA each
          const int64_t n = std::max<int64_t>(1, std::min<int64_t>(g.tiles, int64_t(double(g.tiles) / avg + 0.5)));
          for (int32_t k = 0; k < g.n; k++)
            for (int64_t j = 0; j < n; j++) {
              const int64_t tb0 = g.tiles * j / n, tb1 = g.tiles * (j + 1) / n;
              add_item(g.first + k, tb0 * kUniqTileRows, std::min(rows, tb1 * kUniqTileRows));
              P->uitems.back().count_surv = (count_first && k == 0) ? 1 : 0;
              P->u_cta_item.push_back(int32_t(P->uitems.size()));
            }
        } else {
          // whole slabs packed into CTAs of about avg tiles
          int64_t acc = 0;
          for (int32_t k = 0; k < g.n; k++) {
            add_item(g.first + k, 0, rows);
            P->uitems.back().count_surv = (count_first && k == 0) ? 1 : 0;
            acc += g.tiles;
            if (double(acc) >= avg || k == g.n - 1) {
              P->u_cta_item.push_back(int32_t(P->uitems.size()));
              acc = 0;
            }
          }
        }
        if (count_first) counted[g.t] = true;
      }
    }
  }
  // work of an item ~ units (tiles or count chunks) * (pairs hashed per unit + 1); CTAs
  // proportional to work, >= 1, <= units.  Aggregated items hash distinct keys only
  // (counted as a quarter of their chunk's slots).
  struct Raw {
    int32_t t, b, e, agg;
    int64_t units;
    double work;
  };
  std::vector<Raw> raw;
  double total = 0;
  for (int32_t t = 0; t < n_tables; t++) {
    const cmp_table& tb = tables[t];
    const int32_t tp = tb.n_sketches * d;
    const int64_t tiles = (tb.n_rows + R - 1) / R;
    if (tiles == 0) continue;
    const int32_t n_slabs = tp ? (tp + s.pairs_per_slab - 1) / s.pairs_per_slab : 1;
    for (int32_t k = 0; k < n_slabs; k++) {
      const int32_t b = k * s.pairs_per_slab, e = std::min(tp, (k + 1) * s.pairs_per_slab);
      int32_t row_pairs = 0, agg_pairs = 0;
      for (int32_t p = b; p < e; p++) {
        const int c = tb.key_col[p / d];
        if ((P->uniq_mask[t] >> c) & 1u) continue;
        if (P->col_agg[t][c] < 0) row_pairs++;
        else agg_pairs++;
      }
      // a slab whose pairs are all hashed by the unique-key kernel, of a table whose
      // survivors are counted elsewhere, has no work here (aggregated pairs may fall back
      // to this kernel at run time, so their slabs stay)
      if (row_pairs == 0 && agg_pairs == 0 && P->surv_by[t] != kSurvRow) continue;
      Raw r{t, b, e, -1, tiles, double(tiles) * double(row_pairs + 1)};
      total += r.work;
      raw.push_back(r);
    }
  }
  // hashing pass of the aggregated columns: chunks of kHashChunk count-array slots
  P->hash_total_chunks = 0;
  P->hash_max_pairs = 1;
  for (AggCol& ac : P->aggs) {
    ac.hash_chunk0 = P->hash_total_chunks;
    if (ac.kind == kAggPresence) continue;  // hashed by the dense kernel
    P->hash_total_chunks += (ac.cap + kHashChunk - 1) / kHashChunk;
    int32_t np = 0;
    for (int32_t k = 0; k < tables[ac.table].n_sketches; k++) np += tables[ac.table].key_col[k] == ac.col ? d : 0;
    P->hash_max_pairs = std::max(P->hash_max_pairs, np);
  }
  P->hash_grid = int32_t(std::min<int64_t>(P->hash_total_chunks, int64_t(sm_count()) * 2));  // resident: 2 per SM
  // dense kernel: slabs of each presence column's pairs (as for the unique-key kernel);
  // each slab's domain split into items of whole runs, about equal work (keys x pairs) per
  // CTA, one CTA per SM; consecutive items of a CTA share a slab where they can
  P->dslabs.clear();
  P->ditems.clear();
  P->d_cta_item.assign(1, 0);
  P->d_words = 0;
  P->n_presence = 0;
  {
    double total = 0;
    for (int32_t ai = 0; ai < int32_t(P->aggs.size()); ai++) {
      const AggCol& ac = P->aggs[ai];
      if (ac.kind != kAggPresence) continue;
      P->n_presence++;
      const cmp_table& tb = tables[ac.table];
      std::vector<int32_t> pairs;
      for (int k = 0; k < tb.n_sketches; k++)
        if (tb.key_col[k] == ac.col)
          for (int i = 0; i < d; i++) pairs.push_back(k * d + i);
      const int max_pps = P->u_pack16 ? 1
                                       : int(std::max<size_t>(1, std::min<size_t>(kUniqMaxPairs,
                                                                                  kUniqSmemBudget / (size_t(w) * 4))));
      const int n_sl = int((pairs.size() + max_pps - 1) / max_pps);
      const int pps = int((pairs.size() + n_sl - 1) / n_sl);
      for (size_t b = 0; b < pairs.size(); b += pps) {
        UniqSlab sl;
        std::memset(&sl, 0, sizeof(sl));
        sl.table = ac.table;
        sl.col = ac.col;
        sl.pad = ai;
        sl.n_pairs = int32_t(std::min(pairs.size() - b, size_t(pps)));
        for (int q = 0; q < sl.n_pairs; q++) sl.pair[q] = pairs[b + q];
        P->d_words = std::max<int32_t>(P->d_words, P->u_pack16 ? int32_t((w + 1) / 2) : sl.n_pairs * w);
        total += double(ac.cap) * sl.n_pairs;
        P->dslabs.push_back(sl);
      }
    }
    if (!P->dslabs.empty()) {
      const int32_t G = sm_count();
      const double per_cta = total / G;
      // items: each slab's runs cut wherever a CTA's share of the total work ends
      double acc = 0;  // work before the current item
      int32_t cta = 0;
      for (int32_t si = 0; si < int32_t(P->dslabs.size()); si++) {
        const UniqSlab& sl = P->dslabs[si];
        const int64_t runs = (P->aggs[sl.pad].cap + kDenseRun - 1) / kDenseRun;
        const double wpr = double(kDenseRun) * sl.n_pairs;  // work per run
        int64_t r = 0;
        while (r < runs) {
          // runs left in CTA `cta`'s share
          const double room = double(cta + 1) * per_cta - acc;
          int64_t take = cta == G - 1 ? runs - r : std::max<int64_t>(1, int64_t(room / wpr + 0.5));
          take = std::min(take, runs - r);
          UniqItem it;
          it.slab = si;
          it.count_surv = 0;
          it.row_begin = r * kDenseRun;
          it.row_end = (r + take) * kDenseRun;
          P->ditems.push_back(it);
          acc += double(take) * wpr;
          r += take;
          if (cta < G - 1 && acc >= double(cta + 1) * per_cta - 0.5 * wpr) {
            P->d_cta_item.push_back(int32_t(P->ditems.size()));
            cta++;
          }
        }
      }
      if (P->d_cta_item.back() != int32_t(P->ditems.size())) P->d_cta_item.push_back(int32_t(P->ditems.size()));
    }
  }
  const double target = double(sm_count()) * ctas_per_sm * 4.0;
  P->items.clear();
  P->cta_item.clear();
  for (const Raw& r : raw) {
    int64_t n = int64_t(r.work / std::max(total, 1.0) * target + 0.5);
    n = std::max<int64_t>(1, std::min<int64_t>(n, r.units));
    BuildItem it;
    it.table = r.t;
    it.pair_begin = r.b;
    it.pair_end = r.e;
    it.n_ctas = int32_t(n);
    it.first_cta = int32_t(P->cta_item.size());
    it.pad = 0;
    for (int64_t c = 0; c < n; c++) P->cta_item.push_back(int32_t(P->items.size()));
    P->items.push_back(it);
  }
  // counting pass: one item per table with aggregated columns, its rows as chunks of a
  // multiple of 4 tiles: about 16 chunks per CTA of the resident wave for the largest
  // tables (a CTA's chunk hand-over is a block barrier and an atomic, so chunks are kept
  // long), at most 64 tiles; a persistent grid of about one resident wave takes the chunks
  // in order
  // (tables with a presence column first, so that a split pass completes every bitmap in its
  // first launch)
  P->cnt_items.clear();
  P->cnt_total_chunks = 0;
  auto has_presence = [&](int32_t t) {
    for (int32_t c = 0; c < CMP_MAX_COLS; c++)
      if (P->col_agg[t][c] >= 0 && P->aggs[P->col_agg[t][c]].kind == kAggPresence) return true;
    return false;
  };
  int64_t presence_chunks = 0;
  for (int pass = 0; pass < 2; pass++)
  for (int32_t t = 0; t < n_tables; t++) {
    int ncol = 0;
    for (int32_t c = 0; c < CMP_MAX_COLS; c++) ncol += P->col_agg[t][c] >= 0;
    if (!ncol || has_presence(t) != (pass == 0)) continue;
    CountItem ci;
    ci.table = t;
    ci.pad = 0;
    const int64_t unit = 4 * int64_t(R);
    const int64_t want = tables[t].n_rows / (int64_t(sm_count()) * 2 * 16);
    ci.chunk_rows = unit * std::max<int64_t>(1, std::min<int64_t>(16, want / unit));
    ci.chunk_begin = P->cnt_total_chunks;
    ci.n_chunks = (tables[t].n_rows + ci.chunk_rows - 1) / ci.chunk_rows;
    P->cnt_total_chunks += ci.n_chunks;
    if (pass == 0) presence_chunks += ci.n_chunks;
    P->cnt_items.push_back(ci);
  }
  P->cnt_grid = 0;  // set below, once the unique-key items are known
  // hot-key caches of the counting pass: the most aggregated columns of any table (at most
  // 4 cached), a power-of-two number of slots per column in about 64 KB
  {
    int max_ac = 0;
    for (int32_t t = 0; t < n_tables; t++) {
      int n = 0;
      for (int32_t c = 0; c < CMP_MAX_COLS; c++)
        n += P->col_agg[t][c] >= 0 && P->aggs[P->col_agg[t][c]].kind == kAggCount;
      max_ac = std::max(max_ac, n);
    }
    P->cache_cols = std::min(max_ac, 4);
    int32_t h = 8192;
    while (P->cache_cols && h > 256 && size_t(h) * 8 * size_t(P->cache_cols) > (size_t(64) << 10)) h >>= 1;
    P->cache_slots = P->cache_cols ? h : 256;
  }
  // counting pass: 512-thread CTAs, two per SM; one per SM when the unique-key kernel runs
  // beside it
  P->cnt_grid = int32_t(std::min<int64_t>(P->cnt_total_chunks, int64_t(sm_count()) * (P->uitems.empty() ? 2 : 1)));
  // split pass: when presence bitmaps and other counted tables are both present (and no
  // unique-key kernel wants the place beside the counting pass), the bitmaps are counted
  // first, then the rest with one CTA per SM and the dense kernel beside it
  P->cnt_split = 0;
  P->cnt_grid_b = 0;
  P->d_cut = 1024;
  if (!P->ditems.empty() && P->uitems.empty() && presence_chunks > 0 && presence_chunks < P->cnt_total_chunks) {
    P->cnt_split = presence_chunks;
    P->cnt_grid = int32_t(std::min<int64_t>(presence_chunks, int64_t(sm_count()) * 2));
    P->cnt_grid_b = int32_t(std::min<int64_t>(P->cnt_total_chunks - presence_chunks, int64_t(sm_count())));
    // The dense kernel's share beside the second counting launch: the part it walks while
    // that launch scans (the rest runs after it, two warps per scheduler instead of one).  The
    // scan's time is its columns' bytes at ~4.7 TB/s; the walk beside it advances at ~0.7 of
    // its ~320 G key x row steps/s alone (GB300 measurements of the 1e9-row workload, whose
    // best share, 0.75, this gives).
    double bytes_b = 0, steps = 0;
    for (const CountItem& ci : P->cnt_items) {
      if (ci.chunk_begin < presence_chunks) continue;
      const cmp_table& tb = tables[ci.table];
      uint32_t used = 0;  // referenced columns: aggregated keys and predicates
      for (int32_t c = 0; c < CMP_MAX_COLS; c++)
        if (P->col_agg[ci.table][c] >= 0) used |= 1u << c;
      for (int32_t p = 0; p < tb.n_preds; p++) used |= 1u << tb.preds[p].col;
      for (int32_t c = 0; c < tb.n_cols && c < 32; c++)
        if ((used >> c) & 1u) bytes_b += double(tb.n_rows) * (tb.cols[c].dtype == CMP_I64 ? 8.0 : 4.0);
    }
    for (const UniqSlab& sl : P->dslabs) steps += double(P->aggs[sl.pad].cap) * sl.n_pairs;
    const double share = steps > 0 ? 0.7 * (bytes_b / 4.7e12) / (steps / 3.2e11) : 1.0;
    P->d_cut = int32_t(std::max(1.0, std::min(1024.0, std::round(share * 1024.0))));
  }
  s.grid = int32_t(P->cta_item.size());
  s.ctas_per_slab = 0;
  P->shape = s;
  size_t off = align16(sizeof(BuildPlanHdr));
  off += align16(sizeof(DevTable) * n_tables);
  off += align16(sizeof(BuildItem) * P->items.size());
  off += align16(sizeof(int32_t) * P->cta_item.size());
  off += align16(sizeof(ZeroSpan) * (n_tables + 1));
  off += align16(sizeof(AggCol) * P->aggs.size());
  off += align16(sizeof(CountItem) * P->cnt_items.size());
  off += align16(sizeof(UniqSlab) * P->uslabs.size());
  off += align16(sizeof(UniqItem) * P->uitems.size());
  off += align16(sizeof(int32_t) * P->u_cta_item.size());
  off += align16(sizeof(UniqSlab) * P->dslabs.size());
  off += align16(sizeof(UniqItem) * P->ditems.size());
  off += align16(sizeof(int32_t) * P->d_cta_item.size());
  P->bytes = off;
  return CMP_OK;
}

}  // extern "C"

extern "C" cmp_status cmp_build_plan_bytes(const cmp_table* tables, int32_t n_tables, int32_t d, int32_t w,
                                           const cmp_build_cfg* cfg, size_t* plan_bytes, size_t* ws_bytes) {
  if (!plan_bytes || !ws_bytes) return CMP_EINVAL;
  BuildPlanParts P;
  // edge ids are validated at encode time (n_edges unknown here): accept any non-negative id
  const cmp_status st = plan_layout(tables, n_tables, d, w, cfg, 1 << 30, &P);
  if (st != CMP_OK) return st;
  *plan_bytes = P.bytes;
  *ws_bytes = P.ws_bytes;
  return CMP_OK;
}

extern "C" cmp_status cmp_build_plan_encode(const cmp_table* tables, int32_t n_tables, int32_t d, int32_t w,
                                            int32_t n_edges, int32_t* const* counters_dev_host,
                                            int64_t* survivors_dev, const cmp_build_cfg* cfg, void* plan_host,
                                            size_t plan_bytes) {
  if (!plan_host || !counters_dev_host || !survivors_dev) return CMP_EINVAL;
  BuildPlanParts P;
  cmp_status st = plan_layout(tables, n_tables, d, w, cfg, n_edges, &P);
  if (st != CMP_OK) return st;
  if (plan_bytes < P.bytes) return CMP_EWORKSPACE;
  for (int32_t t = 0; t < n_tables; t++)
    if (tables[t].n_sketches && !counters_dev_host[t]) return CMP_EINVAL;
  unsigned char* base = static_cast<unsigned char*>(plan_host);
  std::memset(base, 0, P.bytes);
  BuildPlanHdr h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kBuildPlanMagic;
  h.version = kBuildPlanVersion;
  h.n_tables = n_tables;
  h.n_items = int32_t(P.items.size());
  h.d = d, h.w = w, h.n_edges = n_edges;
  h.shape = P.shape;
  size_t off = align16(sizeof(BuildPlanHdr));
  h.off_tables = int64_t(off);
  off += align16(sizeof(DevTable) * n_tables);
  h.off_items = int64_t(off);
  off += align16(sizeof(BuildItem) * P.items.size());
  h.off_cta_item = int64_t(off);
  off += align16(sizeof(int32_t) * P.cta_item.size());
  h.off_zero = int64_t(off);
  off += align16(sizeof(ZeroSpan) * (n_tables + 1));
  h.n_agg = int64_t(P.aggs.size());
  h.off_agg = int64_t(off);
  off += align16(sizeof(AggCol) * P.aggs.size());
  h.n_cnt_items = int64_t(P.cnt_items.size());
  h.off_cnt_items = int64_t(off);
  off += align16(sizeof(CountItem) * P.cnt_items.size());
  h.n_uslab = int64_t(P.uslabs.size());
  h.off_uslab = int64_t(off);
  off += align16(sizeof(UniqSlab) * P.uslabs.size());
  h.n_uitems = int64_t(P.uitems.size());
  h.off_uitems = int64_t(off);
  off += align16(sizeof(UniqItem) * P.uitems.size());
  h.off_u_cta = int64_t(off);
  off += align16(sizeof(int32_t) * P.u_cta_item.size());
  h.u_grid = int32_t(P.u_cta_item.size()) - 1;
  h.n_dslab = int64_t(P.dslabs.size());
  h.off_dslab = int64_t(off);
  off += align16(sizeof(UniqSlab) * P.dslabs.size());
  h.n_ditems = int64_t(P.ditems.size());
  h.off_ditems = int64_t(off);
  off += align16(sizeof(UniqItem) * P.ditems.size());
  h.off_d_cta = int64_t(off);
  off += align16(sizeof(int32_t) * P.d_cta_item.size());
  h.d_grid = int32_t(P.d_cta_item.size()) - 1;
  h.d_pack16 = P.u_pack16;
  h.d_words = P.d_words;
  h.n_presence = P.n_presence;
  h.u_pack16 = P.u_pack16;
  h.u_words = P.u_words;
  h.u_tile_rows = kUniqTileRows;
  h.cnt_total_chunks = P.cnt_total_chunks;
  h.cnt_grid = P.cnt_grid;
  h.cnt_split = P.cnt_split;
  h.cnt_grid_b = P.cnt_grid_b;
  h.d_cut = P.d_cut;
  h.cnt_threads = 512;
  h.cnt_cache_slots = P.cache_slots;
  h.cnt_cache_cols = P.cache_cols;
  h.hash_total_chunks = P.hash_total_chunks;
  h.hash_max_pairs = P.hash_max_pairs;
  h.hash_grid = P.hash_grid;
  h.ws_bytes = int64_t(P.ws_bytes);
  h.total_bytes = int64_t(P.bytes);
  std::vector<ZeroSpan> zs;
  for (int32_t t = 0; t < n_tables; t++) {
    DevTable D = to_dev(&tables[t], counters_dev_host[t], survivors_dev + t);
    for (int32_t c = 0; c < CMP_MAX_COLS; c++) D.agg[c] = P.col_agg[t][c];
    D.uniq_mask = P.uniq_mask[t];
    D.surv_by = P.surv_by[t];
    std::memcpy(base + h.off_tables + sizeof(DevTable) * t, &D, sizeof(D));
    const int64_t cb = int64_t(tables[t].n_sketches) * d * w * 4;
    if (cb) zs.push_back(ZeroSpan{counters_dev_host[t], cb});
  }
  zs.push_back(ZeroSpan{survivors_dev, int64_t(n_tables) * 8});
  h.n_zero = int64_t(zs.size());
  std::memcpy(base + h.off_items, P.items.data(), sizeof(BuildItem) * P.items.size());
  std::memcpy(base + h.off_cta_item, P.cta_item.data(), sizeof(int32_t) * P.cta_item.size());
  std::memcpy(base + h.off_zero, zs.data(), sizeof(ZeroSpan) * zs.size());
  if (!P.aggs.empty()) std::memcpy(base + h.off_agg, P.aggs.data(), sizeof(AggCol) * P.aggs.size());
  if (!P.cnt_items.empty())
    std::memcpy(base + h.off_cnt_items, P.cnt_items.data(), sizeof(CountItem) * P.cnt_items.size());
  if (!P.uslabs.empty()) std::memcpy(base + h.off_uslab, P.uslabs.data(), sizeof(UniqSlab) * P.uslabs.size());
  if (!P.uitems.empty()) std::memcpy(base + h.off_uitems, P.uitems.data(), sizeof(UniqItem) * P.uitems.size());
  std::memcpy(base + h.off_u_cta, P.u_cta_item.data(), sizeof(int32_t) * P.u_cta_item.size());
  if (!P.dslabs.empty()) std::memcpy(base + h.off_dslab, P.dslabs.data(), sizeof(UniqSlab) * P.dslabs.size());
  if (!P.ditems.empty()) std::memcpy(base + h.off_ditems, P.ditems.data(), sizeof(UniqItem) * P.ditems.size());
  std::memcpy(base + h.off_d_cta, P.d_cta_item.data(), sizeof(int32_t) * P.d_cta_item.size());
  std::memcpy(base, &h, sizeof(h));
  return CMP_OK;
}

extern "C" cmp_status cmp_sketch_build_batched(const void* plan_host, const void* plan_dev,
                                               const cmp_hash* hash_dev, void* ws_dev, size_t ws_bytes,
                                               int32_t* status_dev, void* stream) {
  if (!plan_host || !plan_dev) return CMP_EINVAL;
  BuildPlanHdr h;
  std::memcpy(&h, plan_host, sizeof(h));
  if (h.magic != kBuildPlanMagic || h.version != kBuildPlanVersion) return CMP_EINVAL;
  if (h.n_edges > 0 && !hash_dev) return CMP_EINVAL;
  if (h.ws_bytes > 0 && (!ws_dev || ws_bytes < size_t(h.ws_bytes))) return CMP_EWORKSPACE;
  const unsigned char* dev = static_cast<const unsigned char*>(plan_dev);
  cudaStream_t cs = as_stream(stream);
  if (launch_zero_spans(reinterpret_cast<const ZeroSpan*>(dev + h.off_zero), int32_t(h.n_zero), cs) != cudaSuccess)
    return CMP_ECUDA;
  BuildArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tables = reinterpret_cast<const DevTable*>(dev + h.off_tables);
  a.items = reinterpret_cast<const BuildItem*>(dev + h.off_items);
  a.cta_item = reinterpret_cast<const int32_t*>(dev + h.off_cta_item);
  a.hash = hash_dev;
  a.status = status_dev;
  a.d = h.d, a.w = h.w, a.n_edges = h.n_edges;
  a.threads = h.shape.threads, a.tile_rows = h.shape.tile_rows, a.map_slots = h.shape.map_slots;
  a.max_pairs = h.shape.max_pairs, a.smem_pairs = h.shape.smem_pairs;
  a.uslab = reinterpret_cast<const UniqSlab*>(dev + h.off_uslab);
  a.uitem = reinterpret_cast<const UniqItem*>(dev + h.off_uitems);
  a.u_cta_item = reinterpret_cast<const int32_t*>(dev + h.off_u_cta);
  a.n_uitems = h.n_uitems;
  a.u_pack16 = h.u_pack16;
  a.u_words = h.u_words;
  a.dslab = reinterpret_cast<const UniqSlab*>(dev + h.off_dslab);
  a.ditem = reinterpret_cast<const UniqItem*>(dev + h.off_ditems);
  a.d_cta_item = reinterpret_cast<const int32_t*>(dev + h.off_d_cta);
  a.n_ditems = h.n_ditems;
  a.d_pack16 = h.d_pack16;
  a.d_words = h.d_words;
  if (h.n_agg > 0) {
    a.agg = reinterpret_cast<const AggCol*>(dev + h.off_agg);
    a.n_agg = int32_t(h.n_agg);
    a.ws = static_cast<unsigned char*>(ws_dev);
    a.cnt_items = reinterpret_cast<const CountItem*>(dev + h.off_cnt_items);
    a.n_cnt_items = int32_t(h.n_cnt_items);
    a.cnt_total_chunks = h.cnt_total_chunks;
    a.hash_total_chunks = h.hash_total_chunks;
    a.hash_max_pairs = h.hash_max_pairs;
    a.cnt_cache_slots = h.cnt_cache_slots;
    a.cnt_cache_cols = h.cnt_cache_cols;
    // the (max, min) key ranges start from zero (decoding as an empty column), so do the
    // chunk counters of the counting and hashing passes after them
    if (cudaMemsetAsync(ws_dev, 0, 16 * size_t(h.n_agg) + 24, cs) != cudaSuccess) return CMP_ECUDA;
    if (launch_agg_zero(a, cs) != cudaSuccess) return CMP_ECUDA;
  }
  const int32_t hash_grid = h.n_agg > 0 ? h.hash_grid : 0;
  const int32_t d_grid = h.n_ditems > 0 ? h.d_grid : 0;
  if (h.cnt_split > 0) {
    // the tables with presence columns, then the others with the dense kernel beside them
    // (its programmatic dependent: one CTA of each per SM, a memory-bound scan beside an
    // integer-bound walk; every bitmap is complete before the second launch starts)
    if (launch_agg_count(a, h.shape.tile_rows, h.cnt_threads, h.cnt_grid, 0, 0, h.cnt_split, cs) != cudaSuccess ||
        launch_presence_check(a, cs) != cudaSuccess ||
        launch_agg_count(a, h.shape.tile_rows, h.cnt_threads, h.cnt_grid_b, 2, h.cnt_split, h.cnt_total_chunks, cs) !=
            cudaSuccess)
      return CMP_ECUDA;
    // the dense kernel: its share beside the counting launch, then the rest with 512 threads
    // (programmatic dependents both: the second takes each SM the first two leave)
    BuildArgs b = a;
    b.dense_part = h.d_cut < 1024 ? 1 : 0;
    b.dense_cut = h.d_cut;
    if (launch_dense(b, d_grid, true, kDenseThreadsBeside, cs) != cudaSuccess) return CMP_ECUDA;
    if (h.d_cut < 1024) {
      b.dense_part = 2;
      if (launch_dense(b, d_grid, true, kDenseThreadsAlone, cs) != cudaSuccess) return CMP_ECUDA;
    }
    if (h.shape.grid > 0 && launch_build(a, h.shape, cs) != cudaSuccess) return CMP_ECUDA;
    return launch_agg_hash(a, hash_grid, cs) == cudaSuccess ? CMP_OK : CMP_ECUDA;
  }
  if (h.n_agg > 0 &&
      launch_agg_count(a, h.shape.tile_rows, h.cnt_threads, h.cnt_grid, 0, 0, h.cnt_total_chunks, cs) != cudaSuccess)
    return CMP_ECUDA;
  // the unique-key kernel right after the counting pass, as its programmatic dependent:
  // one CTA of each per SM, the two overlap (memory-bound scan, integer-bound hashing)
  if (launch_uniq(a, h.u_grid, kUniqThreadsHost, h.u_tile_rows, cs) != cudaSuccess) return CMP_ECUDA;
  if (launch_presence_check(a, cs) != cudaSuccess) return CMP_ECUDA;
  if (h.shape.grid > 0 && launch_build(a, h.shape, cs) != cudaSuccess) return CMP_ECUDA;
  if (launch_agg_hash(a, hash_grid, cs) != cudaSuccess) return CMP_ECUDA;
  // the presence-bitmap columns, beside the hashing of the counted keys when there is one
  // (as its programmatic dependent: both only read what the counting pass wrote)
  return launch_dense(a, d_grid, hash_grid > 0, kDenseThreadsAlone, cs) == cudaSuccess ? CMP_OK : CMP_ECUDA;
}


extern "C" cmp_status cmp_build_plan_stats(const void* plan_host, cmp_build_plan_info* info) {
  if (!plan_host || !info) return CMP_EINVAL;
  BuildPlanHdr h;
  std::memcpy(&h, plan_host, sizeof(h));
  if (h.magic != kBuildPlanMagic || h.version != kBuildPlanVersion) return CMP_EINVAL;
  info->n_tables = h.n_tables;
  info->n_agg = int32_t(h.n_agg);
  info->n_unique_slabs = int32_t(h.n_uslab);
  info->unique_grid = h.n_uitems > 0 ? h.u_grid : 0;
  info->n_unique_items = h.n_uitems;
  info->row_grid = h.shape.grid;
  info->ws_bytes = h.ws_bytes;
  // zeroing; clearing (+ counting when it has chunks) and hashing of the counted keys; the
  // unique-key kernel; the row kernel
  // unique-key kernel; the row kernel; the presence check and the dense kernel
  info->launches = 1 + (h.n_agg > 0 ? 1 + (h.cnt_grid > 0 ? 1 : 0) + (h.cnt_split > 0 ? 1 : 0) + (h.hash_grid > 0 ? 1 : 0) : 0) +
                   (h.n_uitems > 0 && h.u_grid > 0 ? 1 : 0) + (h.shape.grid > 0 ? 1 : 0) +
                   (h.n_ditems > 0 && h.d_grid > 0 ? 2 : 0) +  // the presence check and the dense kernel
                   (h.n_ditems > 0 && h.d_grid > 0 && h.cnt_split > 0 && h.d_cut < 1024 ? 1 : 0);  // its second part
  info->n_presence = h.n_presence;
  return CMP_OK;
}
