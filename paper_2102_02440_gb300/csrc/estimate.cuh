// Internal structures of the estimate path (plan blob and kernel arguments).
#pragma once

#include "internal.cuh"

namespace cmpk {

typedef __int128 i128;
typedef unsigned __int128 u128;

enum { kInOutput = 0, kInLeaf = 1, kInSlot = 2, kInCond = 3, kInCache = 4 };
constexpr int kEstMaxOps = 64;     // operations of one sub-plan (one per non-leaf table)
constexpr int kEstMaxSubIn = 136;  // edge inputs of one sub-plan
constexpr int kEstMaxLevels = 64;  // launch levels of cached subtree messages
constexpr int kEstMaxCond = 3;     // independent cycles of one sub-plan (conditioned edges)

// One edge of a table operation, in the table's ascending edge-id order.
struct EstIn {
  const int32_t* s;      // this table's sketch on the edge, [d][w]
  const uint32_t* abs;   // its presorted magnitudes, [d][w]
  const int32_t* perm;   // its presort permutation, [d][w]
  const int32_t* msk;    // kInLeaf: the leaf neighbour's sketch on the edge, [d][w]
  const int32_t* rk;     // this table's cross ranks from this sketch: [k][d][w], indexed by the other sketch
  int32_t kind;          // kInOutput / kInLeaf / kInSlot / kInCond
  int32_t slot;          // kInSlot: message slot written by the child's operation; kInCache: cached message;
                         // kInCond: the conditioned edge's ordinal (its digit of the conditioning index)
  int32_t suf;           // kInLeaf / kInSlot: suffix-sum array of the sub-plan (item-persistent)
  int32_t tslot;         // this sketch's index within its table (selects rows of another input's rk)
};

// One non-leaf table of a sub-plan's spanning tree (post-order).
struct EstOp {
  int32_t k;         // number of edges (inputs incl. the output edge)
  int32_t p;         // index of the output edge among them, -1 at the root
  int32_t out_slot;  // message slot written (p >= 0); -1 with p >= 0: the job's cached message
  int32_t in_begin;  // first EstIn
  int32_t rank_off;  // first rank table of the op in the item's rank scratch (units of w int32)
  int32_t pad;
};

struct EstSub {
  int32_t op_begin, n_ops;
  int32_t single;     // 1: one table, estimate = exact survivor count
  int32_t n_chunks;   // conditioning chunks per row (1 for trees)
  int64_t item_begin;
  const int64_t* sv;  // single: that table's survivor count (device)
  int32_t cond;       // 1 if a non-tree edge is conditioned
  int32_t tri;        // index of its TriSub (triangle evaluation), else -1
  double scale;       // sampled tables: prod of 1 / rate over the sub-plan's tables, else 1
  int32_t job;        // >= 0: a cached subtree message (its index), not a sub-plan
  int32_t star;       // >= 0: a star of that family, its rows gathered from the family's lattice
  uint32_t sbits;     // star: its leaf edges, bit u = edge u of the family (ascending edge id)
  int32_t split;      // 1: a tree whose only operation is the root; its chunks split the root's
                      // sorted positions (item [c0, c1)), each recomputing the leaf suffix sums
};
constexpr int32_t kRootSplitMinW = 16384;  // widths from which such roots are split
constexpr int32_t kRootSplit = 8;          // chunks of sorted positions per row

// Star families (sub-plans whose only operation is the root joined to leaves, grouped by
// graph and root).  For the family's K leaf edges U (ascending id), sketch row i and the
// edge a that attains the minimum, the lattice holds for every subset V of U \ {a}
//   T_a(V) = sum_r w_a(r) prod_{b in V} f_ab(r),
//   w_a(r) = s_a[pi_a(r)] m_a[pi_a(r)],  f_ab(r) = suffix sum of m_b in b's sorted order from
//   the cross rank of a's position r,
// so that a star over leaf set S has row estimate sum_{a in S} T_a(S \ {a}).  V's bits are
// the positions of U \ {a}: the low k1 bits index the A side, the high k2 bits the B side.
struct StarFam {
  int32_t in_begin, K;      // its K leaf inputs (EstIn, kind kInLeaf)
  int32_t k1, k2, m1, pad;  // k1 + k2 = K - 1; a lattice unit covers 2^m1 A-side subsets
  int64_t suf_off;          // suffix sums: [d][K][w + 1] int64 at star_suf + suf_off
  int64_t t_off;            // lattice: [d][K][2^(K-1)] at star_t + t_off (and star_tf)
  int64_t q_off;            // star_q + q_off: [2^K] the sub-plan of each leaf set, -1: none
};
struct StarUnit {
  int32_t fam, row, a, blk;  // suffix units: a = the leaf b whose suffix sums are built, blk = -1
};
constexpr int kStarThreads = 256;
constexpr int kStarR = 16;        // sorted positions per chunk
constexpr int kStarMaxK2 = 8;     // B side: at most 256 subsets
constexpr int kStarMaxEnt = 4096; // lattice entries per unit (16 per thread)
inline size_t star_smem_bytes() {
  // B[R][256] and A[R][16] int128 with byte flags and float magnitude bounds, f[15][R] and
  // w[R] int64, lane reduction
  return size_t(kStarR) * (1 << kStarMaxK2) * 21 + size_t(kStarR) * 16 * 21 + 15 * kStarR * 8 + kStarR * 8 +
         size_t(kStarThreads) * 17 + 64;
}

struct EstItem {
  int32_t sub, row, c0, c1;  // conditioning values [c0, c1); trees use [0, 1); triangle: columns [c0, c1)
};

// Digit k (base w) of a conditioning index: the bucket of the sub-plan's k-th conditioned
// edge (ascending edge id) when the index runs over all w^rho assignments of its rho edges.
__device__ __forceinline__ int cond_digit(int c, int k, int w) {
  if (c < w) return k == 0 ? c : 0;
  for (int i = 0; i < k; i++) c /= w;
  return c % w;
}

// Triangle sub-plans: the only cycle is U-W-V with the conditioned edge U-V, and every
// other table is a leaf joined to U, V or W.  Each node lists its edges (EstIn, ascending
// edge id; kInCond = the conditioned edge, kInSlot = a triangle edge, kInLeaf = a leaf).
struct TriNode {
  int32_t in_begin, k;  // first EstIn, number of edges
  int32_t ia, ib;       // U, V: edge to W, conditioned edge.  W: edge to U, edge to V
};
struct TriSub {
  TriNode node[3];  // U, V, W
  int32_t sub, pad;
};
constexpr int32_t kTriMaxW = 16384;   // queries and rows are sorted in shared memory
constexpr int32_t kTriMaxLeaves = 16; // leaves per triangle node
constexpr int32_t kTriCols = 256;     // columns per sweep item (one per thread)

// Per triangle row (sub-plan, sketch row) scratch, in bytes, and its regions.
struct TriLayout {
  int64_t hdr, vec, tmp, sg, pre, rkx, rpre, cky, ccol, qs, qr, qpre, gr, gqb, bytes;
};
__host__ __device__ inline int64_t tri_al(int64_t x) { return (x + 255) & ~int64_t(255); }
__host__ __device__ inline TriLayout tri_layout(int32_t w, int32_t max_leaves) {
  const int64_t W1 = int64_t(w) + 1, nl = 3 * int64_t(max_leaves);
  TriLayout L;
  int64_t o = 0;
  L.hdr = o;  o += tri_al(64);
  L.vec = o;  o += tri_al(16 * 6 * int64_t(w));   // phiU psiU phiV psiV f g, bucket order
  L.tmp = o;  o += tri_al(16 * 3 * int64_t(w));   // leaf-term sums of a node message, one per node
  L.sg = o;   o += tri_al(8 * nl * W1);          // leaf suffix sums
  L.pre = o;  o += tri_al(16 * nl * W1);         // leaf "attains the minimum" prefix sums
  L.rkx = o;  o += tri_al(8 * int64_t(w));       // row keys, sorted within batches
  L.rpre = o; o += tri_al(16 * 3 * W1);          // row prefix sums: phi*f, f, phi
  L.cky = o;  o += tri_al(8 * int64_t(w));       // column keys
  L.ccol = o; o += tri_al(16 * 2 * int64_t(w));  // column phi, g
  L.qs = o;   o += tri_al(4 * int64_t(w));       // query clamp ranks on the column side, sorted
  L.qr = o;   o += tri_al(4 * int64_t(w));       // query clamp ranks on the row side, sorted
  L.qpre = o; o += tri_al(16 * 3 * W1);          // query prefix sums: psiR, psiC, psiR*psiC
  L.gr = o;   o += tri_al(4 * (W1 + 1));         // distinct row-side ranks (group boundaries)
  L.gqb = o;  o += tri_al(4 * (W1 + 1));         // first query of each group
  L.bytes = o;
  return L;
}

struct EstPlanHdr {
  uint64_t magic;
  int32_t version, d, w, max_slots, max_in, grid, threads, max_suf, max_rank;
  int64_t n_sub, n_ops, n_in, n_items;
  int64_t off_subs, off_ops, off_in, off_items, total_bytes;
  int64_t scratch_per_cta;  // bytes
  int64_t ws_bytes;
  int64_t n_gen_items;      // items [0, n_gen_items) run the generic kernel
  int64_t n_tri, off_tri;   // triangle sub-plans
  int64_t tri_row_bytes;
  int32_t tri_max_leaves, tri_nch;  // leaves per node (scratch layout), sweep items per row
  // cached subtree messages: jobs, their items (the first of the generic items), and the
  // end of each level's items (level l reads the messages of levels < l only)
  int64_t n_jobs, n_job_items;
  int32_t n_levels, pad;
  int64_t lvl_end[kEstMaxLevels];
  // star families (CMP_EST_STAR_LATTICE): families, units (suffix units first)
  int64_t n_star, off_star, n_star_units, n_star_suf_units, off_star_units;
  int64_t star_suf_words, star_t_entries;  // workspace: int64 suffix sums, lattice entries
  int64_t off_star_q, n_star_q;            // the families' leaf-set -> sub-plan tables (int32)
  // exact tier beyond int128 (wide = 1): every sub-plan planned on the generic path alone
  // (its own arrays when the main plan uses other paths, else the main plan's), evaluated
  // modulo kWideMods primes for the rows found beyond int128, with a magnitude bound
  int32_t wide, wide_qcap;  // wide_qcap: rows the tier can take per call (more stay out of range)
  int64_t wide_off_subs, wide_off_ops, wide_off_in, wide_off_items, wide_n_items;
  int32_t wide_max_slots, wide_max_in, wide_max_suf, wide_grid;
  int64_t wide_scratch_per_cta;
  int32_t wide_unit_cap, pad2;  // (row, conditioning chunk) units the tier can take per call
};
constexpr int32_t kWideQueueMax = 1 << 19;
constexpr int32_t kWideCtasPerSm = 8;  // the tier's generic kernel: 128-thread CTAs, 8 per SM
constexpr int32_t kWideUnitMax = 1 << 20;
// scratch of the exact tier's own grid (its CTA areas reuse the estimate's scratch region and
// extend it to this size when it is smaller)
constexpr int64_t kWideScratchBudget = int64_t(256) << 20;
constexpr uint64_t kEstPlanMagic = 0x434d504553544d54ull;  // "CMPESTMT"
constexpr int32_t kEstPlanVersion = 8;

// Exact tier beyond int128: a row is evaluated modulo kWideMods primes p_j = 2^62 - c_j
// (exact ring arithmetic: the contraction is sums of products of the counters, and the
// min-abs selections depend only on the presorted magnitudes), and once more in double
// rounded upwards on absolute values, a bound on |E|.  When the bound is below 2^kWideBits
// (< P/2, P the product of the primes), E is the unique integer of (-P/2, P/2) with those
// residues (Garner's algorithm).  Rows are reported as kWideLimbs 64-bit two's-complement
// limbs.
constexpr int kWideMods = 16;
constexpr int kWideLimbs = 16;
constexpr int kWideBits = 990;
__host__ __device__ constexpr uint64_t wide_c(int j) {
  return j == 0 ? 57 : j == 1 ? 87 : j == 2 ? 117 : j == 3 ? 143 : j == 4 ? 153 : j == 5 ? 167 : j == 6 ? 171
       : j == 7 ? 195 : j == 8 ? 203 : j == 9 ? 273 : j == 10 ? 287 : j == 11 ? 317 : j == 12 ? 443
       : j == 13 ? 483 : j == 14 ? 495 : 575;
}
__host__ __device__ constexpr uint64_t wide_p(int j) { return (uint64_t(1) << 62) - wide_c(j); }

struct EstArgs {
  const EstSub* subs;
  const EstOp* ops;
  const EstIn* inputs;
  const EstItem* items;
  i128* partial;         // [n_items]
  int32_t* partial_ovf;  // [n_items]
  void* scratch;
  int64_t scratch_per_cta;  // bytes
  int64_t n_items, n_sub;
  int32_t d, w, max_slots, max_in, grid, threads, max_suf, max_rank;
  int32_t* status;
  int64_t n_gen_items;
  const TriSub* tri;
  int64_t n_tri;
  unsigned char* tri_scratch;  // tri_slots rows of tri_row_bytes
  int64_t tri_row_bytes, tri_slots;
  int32_t tri_max_leaves, tri_nch;
  i128* cache;          // [n_jobs][d][w] cached subtree messages, bucket order
  int32_t* cache_ovf;   // [n_jobs][d] 1: the message left int128
  int64_t n_job_items;
  const StarFam* star;
  const StarUnit* star_units;
  int64_t n_star, n_star_units, n_star_suf_units;
  int64_t* star_suf;
  i128* star_t;
  uint8_t* star_tf;     // 1: the lattice entry left int128
  const int32_t* star_q;  // leaf set -> sub-plan, per family (StarFam.q_off)
  // exact tier beyond int128
  int32_t wide;
  const EstSub* wsubs;
  const EstOp* wops;
  const EstIn* winputs;
  const EstItem* witems;
  int64_t wide_n_items;
  int32_t wide_max_slots, wide_max_in, wide_max_suf, wide_grid, wide_qcap, wide_unit_cap;
  int64_t wide_scratch_per_cta;
  uint32_t* wide_queue;   // [0] rows queued, [1] sub-plans queued, [2] units taken, [4..4+qcap) rows, then sub-plans
  int32_t* wide_slot;     // [n_sub * d] queue slot of each row, -1 when it stays in int128
  i128* wide_in;          // [n_sub * d] the int128 rows of sub-plans in the queue
  int32_t* wide_row_start;  // [qcap] first unit of each queued row (its chunks' units follow), -1: none
  uint64_t* wide_units;   // [unit_cap] (queued row << 32 | conditioning chunk); row ~0u: none
  uint64_t* wide_part;    // [unit_cap][kWideMods + 1]: the unit's residues, then its bound (double bits)
  void* wide_scratch;     // wide_grid areas of wide_scratch_per_cta bytes
  // star rows beyond int128 evaluated on their family's lattice in modular arithmetic, per
  // (family, sketch row), [n_star * d] each: rows queued, 1 when the lattice evaluates them,
  // the most primes one of them needs
  uint32_t* wide_star_cnt;
  int32_t* wide_star_on;
  int32_t* wide_star_kmax;
};

// Unit entries of the exact tier: (queued row << 32) | low word; the low word is a
// conditioning chunk, or kUnitLattice: a star row's single unit, which its family's lattice
// fills (the residues summed over its leaves a of T_a(S \ {a}), the largest of their bounds).
constexpr uint32_t kUnitLattice = 0x80000000u;

// A star sub-plan whose leaf set maps to it in its family's table: its queued rows are
// evaluated on the family's lattice in modular arithmetic when enough rows of the (family,
// sketch row) are queued (else by the generic contraction).
__device__ __forceinline__ bool wide_star_row(const EstArgs& A, int64_t q) {
  const int32_t f = A.subs[q].star;
  return f >= 0 && A.star_q[A.star[f].q_off + A.subs[q].sbits] == int32_t(q);
}
// Units of a queued row of sub-plan q: one per conditioning chunk of its generic plan.
__device__ __forceinline__ int wide_row_units(const EstArgs& A, int64_t q) { return max(1, A.wsubs[q].n_chunks); }

// Round-to-nearest-even of (neg ? -1 : 1) * (top * 2^128 + mag) to binary64, from the
// definition: the top 53 significant bits, then half-ulp and sticky bits.
__device__ inline double mag_to_double(bool neg, uint32_t top, u128 mag) {
  if (top == 0 && mag == 0) return 0.0;
  // bit length
  int nb;
  if (top) nb = 129;
  else {
    const uint64_t hi = uint64_t(mag >> 64);
    nb = hi ? 128 - __clzll(hi) : 64 - __clzll(uint64_t(mag));
  }
  double r;
  if (nb <= 53) {
    r = double(uint64_t(mag));
  } else {
    const int sh = nb - 53;  // bits below the kept significand
    u128 sig, rest_mask, rest, half;
    if (top) {  // nb == 129: value = 2^128 + mag
      sig = (u128(1) << 52) | (mag >> 76);
      rest_mask = (u128(1) << 76) - 1;
      rest = mag & rest_mask;
      half = u128(1) << 75;
    } else {
      sig = mag >> sh;
      rest_mask = (u128(1) << sh) - 1;
      rest = mag & rest_mask;
      half = u128(1) << (sh - 1);
    }
    uint64_t s = uint64_t(sig);
    if (rest > half || (rest == half && (s & 1))) s++;
    int e = sh;
    if (s == (1ull << 53)) {
      s >>= 1;
      e++;
    }
    r = ldexp(double(s), e);
  }
  return neg ? -r : r;
}

__device__ inline double i128_to_double(i128 v) {
  const bool neg = v < 0;
  return mag_to_double(neg, 0, neg ? u128(0) - u128(v) : u128(v));
}

cudaError_t launch_presort(const int32_t* C, int64_t n_rows, int32_t w, uint32_t* abs_out, int32_t* perm_out,
                           cudaStream_t st);
cudaError_t launch_presort_large(const int32_t* C, int64_t n_rows, int32_t w, uint32_t* abs_out, int32_t* perm_out,
                                 void* ws, int64_t rows_per_pass, cudaStream_t st);
int64_t presort_padded(int32_t w);
constexpr int32_t kPresortSmemMaxW = 16384;
// Workspace of an encoded plan: per-item partial sums and flags, the cached subtree
// messages and their flags, `grid` per-CTA scratch areas of the generic kernel, then
// `tri_slots` triangle rows.
inline size_t est_cache_bytes(const EstPlanHdr& H) {
  return align16(sizeof(i128) * size_t(H.n_jobs) * size_t(H.d) * size_t(H.w));
}
inline size_t est_star_bytes(const EstPlanHdr& H) {
  return align16(sizeof(i128) * size_t(H.star_t_entries)) + align16(size_t(H.star_t_entries)) +
         align16(sizeof(int64_t) * size_t(H.star_suf_words));
}
// exact tier: queue counters ([0] rows, [1] sub-plans), the queued rows (sub * d + row) and
// sub-plans, each row's queue slot (-1: it stays in int128), the int128 rows of the queued
// sub-plans, per queued row its residues and bound.  Its kernels run after the others and
// reuse their per-CTA and triangle scratch.
inline size_t est_wide_bytes(const EstPlanHdr& H) {
  if (!H.wide) return 0;
  const size_t rows = size_t(H.n_sub) * size_t(H.d);
  return align16(sizeof(uint32_t) * (4 + size_t(H.wide_qcap) + size_t(H.n_sub))) + align16(sizeof(int32_t) * rows) +
         align16(sizeof(i128) * rows) + align16(sizeof(int32_t) * size_t(H.wide_qcap)) +
         align16(sizeof(uint64_t) * size_t(H.wide_unit_cap)) +
         align16(sizeof(uint64_t) * size_t(H.wide_unit_cap) * (kWideMods + 1)) +
         3 * align16(sizeof(int32_t) * size_t(H.n_star) * size_t(H.d));
}
inline size_t est_fixed_bytes(const EstPlanHdr& H) {
  return align16(sizeof(i128) * size_t(H.n_items)) + align16(sizeof(int32_t) * size_t(H.n_items)) +
         est_cache_bytes(H) + align16(sizeof(int32_t) * size_t(H.n_jobs) * size_t(H.d)) + est_star_bytes(H) +
         est_wide_bytes(H);
}
// The scratch region after the fixed part: `grid` per-CTA areas, then `tri_slots` triangle
// rows; the exact tier's kernel, which runs after every other one, reuses the region for
// `wide_ctas` CTA areas of its own (at least one).
inline size_t est_scratch_bytes(const EstPlanHdr& H, int64_t grid, int64_t tri_slots, int64_t wide_ctas) {
  const size_t main = size_t(H.scratch_per_cta) * size_t(grid) + size_t(H.tri_row_bytes) * size_t(tri_slots);
  const size_t wide = H.wide ? size_t(H.wide_scratch_per_cta) * size_t(wide_ctas < 1 ? 1 : wide_ctas) : 0;
  return main > wide ? main : wide;
}
inline size_t est_ws_bytes(const EstPlanHdr& H, int64_t grid, int64_t tri_slots, int64_t wide_ctas) {
  return est_fixed_bytes(H) + est_scratch_bytes(H, grid, tri_slots, wide_ctas);
}
// wide_ctas: the exact tier's grid, the CTA areas est_scratch_bytes reserved for it (>= 1).
inline EstArgs est_args(const EstPlanHdr& H, const unsigned char* pd, unsigned char* ws, int32_t grid,
                        int64_t tri_slots, int32_t* status, int32_t wide_ctas) {
  EstArgs a;
  a.subs = reinterpret_cast<const EstSub*>(pd + H.off_subs);
  a.ops = reinterpret_cast<const EstOp*>(pd + H.off_ops);
  a.inputs = reinterpret_cast<const EstIn*>(pd + H.off_in);
  a.items = reinterpret_cast<const EstItem*>(pd + H.off_items);
  a.partial = reinterpret_cast<i128*>(ws);
  const size_t o_ovf = align16(sizeof(i128) * size_t(H.n_items));
  const size_t o_cache = o_ovf + align16(sizeof(int32_t) * size_t(H.n_items));
  a.partial_ovf = reinterpret_cast<int32_t*>(ws + o_ovf);
  a.cache = reinterpret_cast<i128*>(ws + o_cache);
  a.cache_ovf = reinterpret_cast<int32_t*>(ws + o_cache + est_cache_bytes(H));
  a.n_job_items = H.n_job_items;
  const size_t o_star = o_cache + est_cache_bytes(H) + align16(sizeof(int32_t) * size_t(H.n_jobs) * size_t(H.d));
  a.star = reinterpret_cast<const StarFam*>(pd + H.off_star);
  a.star_units = reinterpret_cast<const StarUnit*>(pd + H.off_star_units);
  a.star_q = reinterpret_cast<const int32_t*>(pd + H.off_star_q);
  a.n_star = H.n_star;
  a.n_star_units = H.n_star_units;
  a.n_star_suf_units = H.n_star_suf_units;
  a.star_t = reinterpret_cast<i128*>(ws + o_star);
  a.star_tf = ws + o_star + align16(sizeof(i128) * size_t(H.star_t_entries));
  a.star_suf = reinterpret_cast<int64_t*>(ws + o_star + align16(sizeof(i128) * size_t(H.star_t_entries)) +
                                          align16(size_t(H.star_t_entries)));
  a.wide = H.wide;
  a.wsubs = reinterpret_cast<const EstSub*>(pd + H.wide_off_subs);
  a.wops = reinterpret_cast<const EstOp*>(pd + H.wide_off_ops);
  a.winputs = reinterpret_cast<const EstIn*>(pd + H.wide_off_in);
  a.witems = reinterpret_cast<const EstItem*>(pd + H.wide_off_items);
  a.wide_n_items = H.wide_n_items;
  a.wide_max_slots = H.wide_max_slots;
  a.wide_max_in = H.wide_max_in;
  a.wide_max_suf = H.wide_max_suf;
  a.wide_grid = 0;  // set below from the scratch region it shares
  a.wide_qcap = H.wide_qcap;
  a.wide_unit_cap = H.wide_unit_cap;
  a.wide_scratch_per_cta = H.wide_scratch_per_cta;
  {
    const size_t o_wide = est_fixed_bytes(H) - est_wide_bytes(H);
    const size_t rows = size_t(H.n_sub) * size_t(H.d);
    const size_t o_slot = o_wide + align16(sizeof(uint32_t) * (4 + size_t(H.wide_qcap) + size_t(H.n_sub)));
    const size_t o_in = o_slot + align16(sizeof(int32_t) * rows);
    const size_t o_start = o_in + align16(sizeof(i128) * rows);
    const size_t o_units = o_start + align16(sizeof(int32_t) * size_t(H.wide_qcap));
    const size_t o_part = o_units + align16(sizeof(uint64_t) * size_t(H.wide_unit_cap));
    const size_t o_scnt = o_part + align16(sizeof(uint64_t) * size_t(H.wide_unit_cap) * (kWideMods + 1));
    const size_t fam_rows = align16(sizeof(int32_t) * size_t(H.n_star) * size_t(H.d));
    a.wide_star_cnt = H.wide ? reinterpret_cast<uint32_t*>(ws + o_scnt) : nullptr;
    a.wide_star_on = H.wide ? reinterpret_cast<int32_t*>(ws + o_scnt + fam_rows) : nullptr;
    a.wide_star_kmax = H.wide ? reinterpret_cast<int32_t*>(ws + o_scnt + 2 * fam_rows) : nullptr;
    a.wide_queue = H.wide ? reinterpret_cast<uint32_t*>(ws + o_wide) : nullptr;
    a.wide_slot = H.wide ? reinterpret_cast<int32_t*>(ws + o_slot) : nullptr;
    a.wide_in = H.wide ? reinterpret_cast<i128*>(ws + o_in) : nullptr;
    a.wide_row_start = H.wide ? reinterpret_cast<int32_t*>(ws + o_start) : nullptr;
    a.wide_units = H.wide ? reinterpret_cast<uint64_t*>(ws + o_units) : nullptr;
    a.wide_part = H.wide ? reinterpret_cast<uint64_t*>(ws + o_part) : nullptr;
    // the exact tier's kernel runs after every other one and reuses their scratch
    a.wide_scratch = H.wide ? ws + est_fixed_bytes(H) : nullptr;
    if (H.wide && H.wide_scratch_per_cta > 0) a.wide_grid = wide_ctas < 1 ? 1 : wide_ctas;
  }
  a.scratch = ws + est_fixed_bytes(H);
  a.scratch_per_cta = H.scratch_per_cta;
  a.n_items = H.n_items;
  a.n_sub = H.n_sub;
  a.d = H.d;
  a.w = H.w;
  a.max_slots = H.max_slots;
  a.max_in = H.max_in;
  a.grid = grid;
  a.threads = H.threads;
  a.max_suf = H.max_suf;
  a.max_rank = H.max_rank;
  a.status = status;
  a.n_gen_items = H.n_gen_items;
  a.tri = reinterpret_cast<const TriSub*>(pd + H.off_tri);
  a.n_tri = H.n_tri;
  a.tri_scratch = ws + est_fixed_bytes(H) + size_t(H.scratch_per_cta) * size_t(grid);
  a.tri_row_bytes = H.tri_row_bytes;
  a.tri_slots = tri_slots;
  a.tri_max_leaves = H.tri_max_leaves;
  a.tri_nch = H.tri_nch;
  return a;
}

cudaError_t launch_estimate(const EstArgs& a, const EstPlanHdr& H, double* est, int64_t* row_est, cudaStream_t st,
                            int64_t* wide_rows = nullptr);
cudaError_t launch_estimate_wide(const EstArgs& a, double* est, int64_t* wide_rows, cudaStream_t st);
cudaError_t launch_estimate_tri(const EstArgs& a, cudaStream_t st);
cudaError_t launch_estimate_star(const EstArgs& a, cudaStream_t st);
cudaError_t launch_cross_ranks(const uint32_t* abs, const int32_t* perm, int32_t k, int32_t d, int32_t w,
                               const int32_t* edge_id, int32_t* ranks, cudaStream_t st);
cudaError_t launch_cross_ranks_multi(const uint32_t* abs, const int32_t* perm, int32_t n_tables, const int32_t* k,
                                     const int32_t* edge_ids, int32_t d, int32_t w, int32_t* ranks, cudaStream_t st);

}  // namespace cmpk
