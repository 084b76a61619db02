// Internal device/host definitions of libcompass (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "compass.h"

namespace cmpk {

// ------------------------------------------------------------------ constants
constexpr uint64_t kP61 = (1ull << 61) - 1;     // Mersenne prime of the CW hash family
constexpr uint32_t kM31 = 0x7FFFFFFFu;
constexpr uint64_t kM30 = (1ull << 30) - 1;
constexpr unsigned long long kEmptyKey = ~0ull;  // never a field element (< 2^61)

// ------------------------------------------------------- arithmetic mod 2^61-1
// A field element v < 2^61 is held as two limbs v = hi * 2^31 + lo (lo < 2^31,
// hi < 2^30) so that every partial product fits 62 bits and three of them can be
// summed in one uint64 before a single Mersenne fold (2^61 = 1, 2^62 = 2 mod p).
struct Limb {
  uint32_t lo, hi;
};

__device__ __forceinline__ Limb limb(uint64_t v) { return {uint32_t(v) & kM31, uint32_t(v >> 31)}; }
__device__ __forceinline__ uint64_t fold61(uint64_t v) { return (v & kP61) + (v >> 61); }
__device__ __forceinline__ uint64_t canon61(uint64_t v) { return v >= kP61 ? v - kP61 : v; }

// key -> residue of the sign-extended key mod p, in [0, p).  For k < 0 write
// k = -1 - m with m = ~k >= 0; then k mod p = p - 1 - (m mod p).
__device__ __forceinline__ uint64_t key_field(int64_t k) {
  const uint64_t s = uint64_t(k >> 63);
  const uint64_t m = uint64_t(k) ^ s;
  const uint64_t y = canon61(fold61(m));  // m < 2^64: fold < p + 8, one subtraction
  return s ? (kP61 - 1 - y) : y;
}

// (a * b) mod p from limbs.  t0 < 2^62, t1 < 2^62, t2 < 2^60 and
// a*b = t2 2^62 + t1 2^31 + t0 = 2 t2 + (t1 >> 30) + (t1 & (2^30-1)) 2^31 + t0 (mod p);
// the sum is < 2^63 + 2^32.
__device__ __forceinline__ uint64_t mulmod61(Limb a, Limb b) {
  const uint64_t t0 = uint64_t(a.lo) * b.lo;
  const uint64_t t1 = uint64_t(a.lo) * b.hi + uint64_t(a.hi) * b.lo;
  const uint64_t t2 = uint64_t(a.hi) * b.hi;
  const uint64_t s = t0 + (t1 >> 30) + ((t1 & kM30) << 31) + 2 * t2;
  return canon61(fold61(s));
}

// Hash parameters of one (edge, row) pre-split into limbs (48 bytes, 16-aligned).
struct __align__(16) PairParam {
  uint32_t a_lo, a_hi, c1_lo, c1_hi, c2_lo, c2_hi, c3_lo, c3_hi;
  uint64_t b, c0;
};

__host__ __device__ inline PairParam make_pair_param(const cmp_hash& h) {
  PairParam q;
  q.a_lo = uint32_t(h.a) & kM31;
  q.a_hi = uint32_t(h.a >> 31);
  q.c1_lo = uint32_t(h.c1) & kM31;
  q.c1_hi = uint32_t(h.c1 >> 31);
  q.c2_lo = uint32_t(h.c2) & kM31;
  q.c2_hi = uint32_t(h.c2 >> 31);
  q.c3_lo = uint32_t(h.c3) & kM31;
  q.c3_hi = uint32_t(h.c3 >> 31);
  q.b = h.b;
  q.c0 = h.c0;
  return q;
}

// Powers of the key, shared by every (sketch, row) that hashes the same key.
struct KeyPow {
  Limb x, x2, x3;
};

__device__ __forceinline__ KeyPow key_powers(uint64_t x) {
  KeyPow k;
  k.x = limb(x);
  const uint64_t x2 = mulmod61(k.x, k.x);
  k.x2 = limb(x2);
  k.x3 = limb(mulmod61(k.x2, k.x));
  return k;
}

// Bucket: ((a x + b) mod p) mod w.  Sum bound: t0 + (t1>>30) + ((t1&M30)<<31) + 2 t2 + b
// < 2^62 + 2^32 + 3 * 2^61 < 2^64.
// SMALLX: the caller guarantees x < 2^31 (k.x.hi == 0), so the products with x.hi, which
// are zero, are left out (same value, fewer multiplies).
template <bool SMALLX = false>
__device__ __forceinline__ uint64_t cw_bucket_residue(const PairParam& q, const KeyPow& k) {
  const uint64_t t0 = uint64_t(q.a_lo) * k.x.lo;
  const uint64_t t1 = SMALLX ? uint64_t(q.a_hi) * k.x.lo : uint64_t(q.a_lo) * k.x.hi + uint64_t(q.a_hi) * k.x.lo;
  const uint64_t t2 = SMALLX ? 0 : uint64_t(q.a_hi) * k.x.hi;
  const uint64_t s = t0 + (t1 >> 30) + ((t1 & kM30) << 31) + 2 * t2 + q.b;
  return canon61(fold61(s));
}
template <bool POW2, bool SMALLX = false>
__device__ __forceinline__ uint32_t cw_bucket(const PairParam& q, const KeyPow& k, uint32_t w) {
  const uint64_t r = cw_bucket_residue<SMALLX>(q, k);
  if (POW2) return uint32_t(r) & (w - 1);
  return uint32_t(r % w);
}

// Sign: parity of (c3 x^3 + c2 x^2 + c1 x + c0) mod p, as +1 / -1.  The three products
// are summed by limb position: S0 < 3 * 2^62, S1 < 6 * 2^61, S2 < 3 * 2^60, and
// fold(S0) + (S1>>30) + ((S1&M30)<<31) + 2 S2 + c0 < 6 * 2^61 + 2^35 < 2^64.
template <bool SMALLX = false>
__device__ __forceinline__ uint64_t cw_sign_residue(const PairParam& q, const KeyPow& k) {
  const uint64_t S0 = uint64_t(q.c1_lo) * k.x.lo + uint64_t(q.c2_lo) * k.x2.lo + uint64_t(q.c3_lo) * k.x3.lo;
  const uint64_t S1 = (SMALLX ? 0 : uint64_t(q.c1_lo) * k.x.hi) + uint64_t(q.c1_hi) * k.x.lo +
                      uint64_t(q.c2_lo) * k.x2.hi + uint64_t(q.c2_hi) * k.x2.lo + uint64_t(q.c3_lo) * k.x3.hi +
                      uint64_t(q.c3_hi) * k.x3.lo;
  const uint64_t S2 = (SMALLX ? 0 : uint64_t(q.c1_hi) * k.x.hi) + uint64_t(q.c2_hi) * k.x2.hi +
                      uint64_t(q.c3_hi) * k.x3.hi;
  const uint64_t v = fold61(S0) + (S1 >> 30) + ((S1 & kM30) << 31) + 2 * S2 + q.c0;
  return canon61(fold61(v));
}
template <bool SMALLX = false>
__device__ __forceinline__ int cw_sign(const PairParam& q, const KeyPow& k) {
  return 1 - 2 * int(cw_sign_residue<SMALLX>(q, k) & 1);
}

// ---- Horner form (one (sketch, row) pair per key: no powers to share).  The same two
// residues, (a x + b) mod p and (c3 x^3 + c2 x^2 + c1 x + c0) mod p = ((c3 x + c2) x + c1) x
// + c0, with intermediates kept only partly reduced: every step's result y satisfies
// y < 2^61 + 5 and y = the exact residue (mod p).
struct KeyX {
  uint32_t lo, hi, hi2;  // x < p as lo + hi 2^31 (lo < 2^31, hi < 2^30), hi2 = 2 hi
};
__device__ __forceinline__ KeyX key_x(uint64_t x) {
  return {uint32_t(x) & kM31, uint32_t(x >> 31), uint32_t(x >> 30) & ~1u};
}

// y x + c folded once, for y < 2^61 + 8 given as (ylo < 2^31, yhi <= 2^30), x < p, c < 2^61.
// y x = ylo xlo + (ylo xhi + yhi xlo) 2^31 + yhi xhi 2^62 and 2^62 = 2, 2^61 = 1 (mod p), so with
// t1 = ylo xhi + yhi xlo (< 2^62 + 2^31):
//   y x + c = ylo xlo + yhi (2 xhi) + c + (t1 >> 30) + (t1 & (2^30-1)) 2^31   (mod p),
// a sum below 2^62 + 2^61 + 2^61 + 2^33 + 2^61 < 2^64; one fold leaves it below 2^61 + 5.
// SMALLX: x < 2^31 (xhi = 0), the products with xhi are zero and left out.
template <bool SMALLX>
__device__ __forceinline__ uint64_t mul_add_fold(uint32_t ylo, uint32_t yhi, const KeyX& x, uint64_t c) {
  const uint64_t t1 = SMALLX ? uint64_t(yhi) * x.lo : uint64_t(ylo) * x.hi + uint64_t(yhi) * x.lo;
  const uint64_t s = uint64_t(ylo) * x.lo + (SMALLX ? 0 : uint64_t(yhi) * x.hi2) + c + (t1 >> 30) +
                     ((t1 & kM30) << 31);
  return fold61(s);
}

// The same step for x < 2^31 (xhi = 0) with every product, shift and add on the multiply
// pipe: with t1 = yhi xlo (< 2^61: yhi <= 2^30) split as t1hi 2^32 + t1lo,
//   t1 2^31 = t1hi 2^63 + t1lo 2^31 = 4 t1hi + t1lo 2^31   (mod p, 2^63 = 4 2^61),
// so y x + c = ylo xlo + c + t1lo 2^31 + 4 t1hi (mod p), a sum below 2^62 + 2^61 + 2^63 +
// 2^31 < 2^64, folded once.  m31 = 2^31 and m4 = 4 come in as run-time values so that the
// compiler keeps them as multiplications.
__device__ __forceinline__ uint64_t mul_add_fold_sx(uint32_t ylo, uint32_t yhi, uint32_t xlo, uint64_t c,
                                                    uint32_t m31, uint32_t m4) {
  const uint64_t t1 = uint64_t(yhi) * xlo;
  uint64_t s = uint64_t(ylo) * xlo + c;
  s += uint64_t(uint32_t(t1)) * m31;
  s += uint64_t(uint32_t(t1 >> 32)) * m4;
  return fold61(s);
}

// For y < 2^61 + 8: 1 if y >= p (its residue is then y - p), else 0.
__device__ __forceinline__ uint32_t ge_p(uint64_t y) { return uint32_t((y + 1) >> 61); }

// Bucket ((a x + b) mod p) mod w; the same value as cw_bucket.  For w a power of two (w <=
// 2^31 divides 2^61), y - p = y + 1 (mod w).
template <bool POW2, bool SMALLX>
__device__ __forceinline__ uint32_t cw_bucket_h(const PairParam& q, const KeyX& x, uint32_t w, uint32_t m31 = 0,
                                                uint32_t m4 = 0) {
  const uint64_t y = SMALLX ? mul_add_fold_sx(q.a_lo, q.a_hi, x.lo, q.b, m31, m4)
                            : mul_add_fold<false>(q.a_lo, q.a_hi, x, q.b);
  if (POW2) return (uint32_t(y) + ge_p(y)) & (w - 1);
  return uint32_t((ge_p(y) ? y - kP61 : y) % w);
}

// Sign: parity of ((c3 x + c2) x + c1) x + c0 mod p, as +1 / -1; the same value as cw_sign.
// The residue of the last y is y - p when y >= p, whose parity is flipped (p is odd).
template <bool SMALLX>
__device__ __forceinline__ int cw_sign_h(const PairParam& q, const KeyX& x, uint64_t c2, uint64_t c1,
                                         uint32_t m31 = 0, uint32_t m4 = 0) {
  uint64_t y;
  if (SMALLX) {
    y = mul_add_fold_sx(q.c3_lo, q.c3_hi, x.lo, c2, m31, m4);
    y = mul_add_fold_sx(uint32_t(y) & kM31, uint32_t(y >> 31), x.lo, c1, m31, m4);
    y = mul_add_fold_sx(uint32_t(y) & kM31, uint32_t(y >> 31), x.lo, q.c0, m31, m4);
  } else {
    y = mul_add_fold<false>(q.c3_lo, q.c3_hi, x, c2);
    y = mul_add_fold<false>(uint32_t(y) & kM31, uint32_t(y >> 31), x, c1);
    y = mul_add_fold<false>(uint32_t(y) & kM31, uint32_t(y >> 31), x, q.c0);
  }
  return 1 - 2 * int((uint32_t(y) ^ ge_p(y)) & 1u);
}

// Output r (0-based) of SplitMix64 (Steele, Lea & Flood 2014) seeded with `seed`: the
// generator's state after r + 1 steps, through its finaliser.
__host__ __device__ inline uint64_t splitmix64_at(uint64_t seed, uint64_t r) {
  uint64_t z = seed + (r + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Sample threshold of a rate: 0 (no sample) for 0 or 1, else floor(rate * 2^64), at least 1.
inline uint64_t sample_keep_of(double rate) {
  if (!(rate > 0.0 && rate < 1.0)) return 0;
  const uint64_t k = uint64_t(rate * 18446744073709551616.0);
  return k ? k : 1;
}

// ------------------------------------------------------------ build structures
struct DevPred {
  int32_t col, op;
  int64_t lo, hi;
  const uint32_t* bitmap;
  int64_t nbits;
};

struct DevTable {
  int64_t n_rows;
  int32_t n_cols, n_preds, n_sketches;
  int32_t vec_ok;  // every column 16-byte aligned: 128-bit loads allowed
  int32_t filtered;  // predicates or a row sample: tiles go through the survivor compaction
  int32_t surv_by;   // batched build: kernel that counts the survivors (kSurvRow / kSurvCount / kSurvUniq)
  uint64_t sample_seed, sample_keep;  // row r is sampled iff splitmix64_at(seed, r) < keep (keep 0: no sample)
  const void* col[CMP_MAX_COLS];
  int32_t dtype[CMP_MAX_COLS];
  DevPred pred[CMP_MAX_PREDS];
  int32_t key_col[CMP_MAX_SKETCHES];
  int32_t edge_id[CMP_MAX_SKETCHES];
  int32_t* counters;   // [n_sketches][d][w]
  int64_t* survivors;  // one int64
  int32_t agg[CMP_MAX_COLS];  // batched build: AggCol index of each aggregated key column, else -1
  uint32_t uniq_mask;         // batched build: key columns hashed by the unique-key kernel (bit c)
  int32_t pad1;
};
enum { kSurvRow = 0, kSurvCount = 1, kSurvUniq = 2 };

// Key aggregation of the batched build.  A key column of a large table is reduced to one
// (key, survivor count) entry per distinct key before hashing: the Fast-AGMS update is
// linear and the int32 counters wrap exactly, so count * xi(key) added once per entry
// gives the counters of one update per tuple.  The counting pass adds each surviving key
// to slot (key - base) & mask of the column's count array (cap slots, cleared before the
// pass) and records the smallest and largest surviving key.  Two layouts:
//  - declared domain [base, base + cap): mask = ~0; a key outside it marks the column as
//    out of range (its counts are then discarded);
//  - no declaration: cap is a power of two and mask = cap - 1, so any cap consecutive
//    keys occupy distinct slots.
// After the pass, a column whose surviving keys span at most cap values is "active" and
// its entries are hashed by k_agg_hash; otherwise it keeps the per-row path.  Workspace:
// [n_agg] x (max, min) encoded as uint64 pairs, then the chunk counters of the counting
// and hashing passes (two uint64; all zeroed before each build, 256-aligned area), then
// each column's int32 count array at byte offset `off`.
// A third kind, the presence bitmap, serves a unique key column with a declared domain in
// a table without predicates: the counting pass sets bit (key - base) of a bitmap instead
// of counting, and k_dense_hash walks the domain in key order.  A key outside the domain
// makes the column inactive, and so does a bitmap with fewer set bits than the table has
// rows (a key seen twice: the column is not unique after all), checked by
// k_presence_check; an inactive column keeps the per-row path.  After the bitmap's whole
// runs, its allocation holds the check's set-bit total and CTA ticket (PresenceCheck).
enum { kAggCount = 0, kAggPresence = 1 };
struct AggCol {
  int32_t table, col;
  int64_t cap;   // count slots (presence: domain keys)
  int64_t off;   // byte offset of the count array (presence: the bitmap) in the workspace
  int64_t base;  // key of slot 0 (declared domain) or 0
  uint64_t mask; // ~0 (declared domain) or cap - 1 (power of two)
  int64_t hash_chunk0;  // first chunk of this column in the hashing pass (kHashChunk slots each)
  int32_t kind, pad;    // kAggCount / kAggPresence
};
constexpr int64_t kHashChunk = 16384;
// Presence bitmaps are walked in runs of kDenseRun keys (8 words); a bitmap holds whole runs.
constexpr int64_t kDenseRun = 256;
__host__ __device__ inline int64_t presence_words(int64_t cap) { return (cap + kDenseRun - 1) / kDenseRun * (kDenseRun / 32); }
struct PresenceCheck {
  unsigned long long bits;  // set bits counted so far
  unsigned int ticket;      // CTAs done
  unsigned int pad;
};

// Order-preserving maps of an int64 to uint64, for atomicMax on the stats pairs (both
// zero-initialised: an empty column decodes as max < min).
__host__ __device__ inline uint64_t enc_max(int64_t v) { return uint64_t(v) ^ (1ull << 63); }
__host__ __device__ inline uint64_t enc_min(int64_t v) { return ~(uint64_t(v) ^ (1ull << 63)); }
__host__ __device__ inline int64_t dec_max(uint64_t e) { return int64_t(e ^ (1ull << 63)); }
__host__ __device__ inline int64_t dec_min(uint64_t e) { return int64_t(~e ^ (1ull << 63)); }

// Whether aggregated column `a` (index ai) takes the aggregated path in this run (read
// after the counting pass), with its smallest surviving key and key range.
__device__ __forceinline__ bool agg_active(const AggCol& a, int ai, const unsigned char* ws, int64_t* kmin,
                                           int64_t* range) {
  const unsigned long long* st = reinterpret_cast<const unsigned long long*>(ws) + 2 * int64_t(ai);
  const int64_t mx = dec_max(st[0]), mn = dec_min(st[1]);
  if (mx < mn) return false;
  const uint64_t r = uint64_t(mx) - uint64_t(mn);
  if (r >= uint64_t(a.cap)) return false;
  *kmin = mn;
  *range = int64_t(r) + 1;
  return true;
}

// Unique key columns (declared distinct, e.g. primary keys) of the batched build: no key
// repeats, so aggregation cannot reduce the hashing.  k_uniq_hash hashes each surviving
// row once per (sketch, row) pair with a slab of the column's pairs held in shared
// memory.  A slab is up to kUniqMaxPairs pairs of one column; an item is one slab over a
// range of the table's rows.
constexpr int32_t kUniqMaxPairs = 32;
struct UniqSlab {
  int32_t table, col, n_pairs, pad;
  int32_t pair[kUniqMaxPairs];  // pair = sketch * d + row of the table
};
struct UniqItem {
  int32_t slab, count_surv;  // count_surv: this item adds its range's survivors to the table's count
  int64_t row_begin, row_end;
};
// k_dense_hash reuses both: a slab's pad is the AggCol index of its presence column, and an
// item's [row_begin, row_end) is a range of domain offsets (key - base), whole runs.

// One (table, slab of (sketch,row) pairs) handled by n_ctas consecutive CTAs walking tiles
// of the table's rows (aggregated key columns are hashed by k_agg_hash instead).
struct BuildItem {
  int32_t table;
  int32_t pair_begin, pair_end;
  int32_t n_ctas;
  int32_t first_cta;
  int32_t pad;
};

// Counting pass of key aggregation: the rows of one table as chunks [chunk_begin,
// chunk_begin + n_chunks) of the pass's global chunk sequence (chunk_rows each), handed out
// to the persistent CTAs in order by an atomic counter.
struct CountItem {
  int32_t table, pad;
  int64_t chunk_begin, n_chunks;
  int64_t chunk_rows;  // a multiple of 4 tiles
};

struct BuildShape {
  int32_t mode;            // 1 smem, 2 global
  int32_t dedupe;          // 0 / 1
  int32_t threads;
  int32_t tile_rows;
  int32_t map_slots;       // power of two >= 2 * tile_rows (dedupe only)
  int32_t max_pairs;       // max pairs of any item (sizes the parameter area)
  int32_t smem_pairs;      // pairs whose counters live in shared memory (mode 1)
  int32_t pairs_per_slab;  // single-table launches
  int32_t ctas_per_slab;   // single-table launches
  int32_t grid;
  size_t smem_bytes;
};

struct BuildArgs {
  DevTable table;             // single-table launch (items == nullptr)
  const DevTable* tables;     // batched launch
  const BuildItem* items;
  const int32_t* cta_item;    // [grid] item of each CTA
  const cmp_hash* hash;       // [n_edges * d]
  int32_t* status;
  int32_t d, w, n_edges;
  int32_t threads, tile_rows, map_slots, max_pairs, smem_pairs;
  int32_t pairs_per_slab, ctas_per_slab;
  const AggCol* agg;  // key aggregation (batched build only)
  int32_t n_agg;
  unsigned char* ws;
  const CountItem* cnt_items;
  int32_t n_cnt_items;
  int32_t cnt_work_slot;                      // chunk counter of this launch of the counting pass
  int64_t cnt_chunk_begin, cnt_chunk_end;     // its chunks
  int32_t cnt_cache_slots, cnt_cache_cols;  // counting pass: hot-key cache slots per column, columns cached
  int64_t cnt_total_chunks;
  int64_t hash_total_chunks;  // hashing pass of the aggregated columns
  int32_t hash_max_pairs;     // most (sketch, row) pairs on one aggregated column
  // unique-key kernel
  const UniqSlab* uslab;
  const UniqItem* uitem;
  const int32_t* u_cta_item;  // [grid + 1] first item of each CTA
  int64_t n_uitems;
  int32_t u_pack16;  // 1: one pair per slab, counters as two 16-bit halves per word
  int32_t u_words;   // shared-memory counter words of a slab
  uint32_t m31, m4;  // 2^31 and 4 (multipliers of the Horner steps)
  // dense (presence-bitmap) kernel: slabs, items and CTA map as for the unique-key kernel
  const UniqSlab* dslab;
  const UniqItem* ditem;
  const int32_t* d_cta_item;
  int64_t n_ditems;
  int32_t d_pack16, d_words;
  // the dense kernel's share of each item's runs: 0 all; 1 the first ceil(n d_cut / 1024);
  // 2 the rest
  int32_t dense_part, dense_cut;
};

// Plan blob (host-encoded, device-read) for the batched build.
struct BuildPlanHdr {
  uint64_t magic;
  int32_t version, n_tables, n_items, d, w, n_edges;
  BuildShape shape;
  int64_t off_tables, off_items, off_cta_item, off_zero, n_zero;  // byte offsets in the blob
  int64_t total_bytes;
  int64_t n_agg, off_agg;                            // aggregated key columns
  int64_t n_cnt_items, off_cnt_items, cnt_total_chunks;  // counting pass
  int32_t cnt_grid, cnt_threads;
  int64_t ws_bytes;
  int32_t cnt_cache_slots, cnt_cache_cols;
  int64_t hash_total_chunks;
  int32_t hash_max_pairs, hash_grid;
  int64_t n_uslab, off_uslab, n_uitems, off_uitems, off_u_cta;  // unique-key kernel
  int32_t u_grid, u_pack16, u_words, u_tile_rows;
  int64_t n_dslab, off_dslab, n_ditems, off_ditems, off_d_cta;  // dense kernel
  int32_t d_grid, d_pack16, d_words, n_presence;
  // counting pass in two launches (cnt_split > 0): chunks [0, cnt_split) of the tables with
  // presence columns first, then [cnt_split, total) with the dense kernel beside it
  int64_t cnt_split;
  // split pass: the dense kernel walks the first d_cut / 1024 of each item's runs beside the
  // second counting launch, the rest after it with 512 threads (d_cut = 1024: all beside)
  int32_t cnt_grid_b, d_cut;
};
constexpr int32_t kBuildPlanVersion = 10;
struct ZeroSpan {
  void* ptr;
  int64_t bytes;
};
constexpr uint64_t kBuildPlanMagic = 0x434d504255494c44ull;  // "CMPBUILD"

// Fire-and-forget atomic additions (PTX red, relaxed): the same update as atomicAdd, with
// no result register, so no instruction waits for the reply.
__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add(int32_t* p, int32_t v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(int32_t* p, int32_t v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(uint32_t(__cvta_generic_to_shared(p))), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(uint32_t* p, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(uint32_t(__cvta_generic_to_shared(p))), "r"(v) : "memory");
}

// device status helper: first error wins
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// launchers implemented in the .cu files
size_t build_smem_bytes(const BuildShape& s, int w);
cudaError_t launch_build(const BuildArgs& a, const BuildShape& s, cudaStream_t st);
size_t agg_count_smem_bytes(int32_t tile_rows, int32_t cache_slots, int32_t cache_cols, int32_t threads);
cudaError_t launch_agg_zero(const BuildArgs& a, cudaStream_t st);
cudaError_t launch_presence_check(const BuildArgs& a, cudaStream_t st);
cudaError_t launch_agg_count(const BuildArgs& a, int32_t tile_rows, int32_t cnt_threads, int32_t cnt_grid,
                             int32_t work_slot, int64_t chunk_begin, int64_t chunk_end, cudaStream_t st);
size_t uniq_smem_bytes(int32_t words, int32_t tile_rows);
cudaError_t launch_uniq(const BuildArgs& a, int32_t grid, int32_t threads, int32_t tile_rows, cudaStream_t st);
cudaError_t launch_zero_spans(const ZeroSpan* spans_dev, int32_t n, cudaStream_t st);
cudaError_t launch_agg_hash(const BuildArgs& a, int32_t grid, cudaStream_t st);
size_t dense_smem_bytes(int32_t words);
cudaError_t launch_dense(const BuildArgs& a, int32_t grid, bool pdl, int32_t threads, cudaStream_t st);
constexpr int32_t kDenseThreadsAlone = 512, kDenseThreadsBeside = 256;

int sm_count();
size_t smem_optin_bytes();
// host checks and device descriptor of one cmp_table (api_build.cu)
cmp_status check_table(const cmp_table* t, int32_t d, int32_t w, int32_t n_edges);
DevTable to_dev(const cmp_table* t, int32_t* counters, int64_t* survivors);

}  // namespace cmpk
