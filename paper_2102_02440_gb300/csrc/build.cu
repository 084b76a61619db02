// Push-down selection fused with the Fast-AGMS sketch update (Sec. 2 "Partitioned query
// execution", Sec. 3.2 "Fast-AGMS Sketches").
//
// One CTA owns a slab: a contiguous range of (sketch, row) pairs of one table.  In
// mode 1 the slab's counters are privatised in shared memory (int32, exact), in mode 2
// (w too large for shared memory) updates go to the L2-resident global counters.  The
// CTA walks tiles of the table's rows:
//   A. predicate pass: 128-bit loads of the predicate columns, conjunction, warp-ballot
//      compaction of the surviving row offsets into shared memory;
//   B. per key column of the slab: optional aggregation of equal keys of the tile in a
//      shared-memory hash map (the update is linear, so count * xi is exact), then for
//      every distinct key and every pair of the slab on that column the CW bucket and
//      sign, and one shared-memory (or L2) atomic add;
//   C. after the last tile: the private counters are added into the final sketch with
//      one global atomic per nonzero counter (partial sketches merge by addition,
//      Sec. 2 "Sketches").
// The kernel has no inter-CTA waits.
//
// Key aggregation (batched build, large tables): before the build kernel, k_agg_zero
// clears each aggregated key column's count array and k_agg_count counts the survivors
// per key: each CTA keeps a shared-memory cache of the keys it meets first (the frequent
// keys of a skewed column settle there), counts them there and every other key with one
// global atomic, adds its cache to the count arrays at the end, and records the range of
// the surviving keys.  After the build kernel, k_agg_hash hashes each nonzero (key,
// count) entry once per pair instead of once per tuple; the build kernel's row items skip
// those columns.  Columns declared unique are hashed by k_uniq_hash (build_unique.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "tile.cuh"

namespace cmpk {

namespace {

__device__ __forceinline__ uint32_t map_slot(uint64_t x, uint32_t mask) {
  return uint32_t((x * 0x9E3779B97F4A7C15ull) >> 40) & mask;
}

constexpr int kMaxSlotsPerThread = 8;

}  // namespace

template <bool GLOBAL, bool DEDUPE, bool POW2>
__global__ void __launch_bounds__(1024) k_sketch_build(const __grid_constant__ BuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;

  // ---- resolve the work item of this CTA
  const DevTable* tb;
  int pair_begin, pair_end, cta_in_slab, n_ctas;
  if (A.items) {
    const BuildItem it = A.items[A.cta_item[blockIdx.x]];
    tb = A.tables + it.table;
    pair_begin = it.pair_begin;
    pair_end = it.pair_end;
    cta_in_slab = int(blockIdx.x) - it.first_cta;
    n_ctas = it.n_ctas;
  } else {
    tb = &A.table;
    const int slab = int(blockIdx.x) / A.ctas_per_slab;
    cta_in_slab = int(blockIdx.x) % A.ctas_per_slab;
    n_ctas = A.ctas_per_slab;
    pair_begin = slab * A.pairs_per_slab;
    const int total_pairs = tb->n_sketches * A.d;
    pair_end = min(pair_begin + A.pairs_per_slab, total_pairs);
  }
  // Key columns of the slab hashed elsewhere: by the unique-key kernel (declared unique),
  // or by the aggregated path when their counting pass found them in range.  If every key
  // column of the slab is hashed elsewhere and the survivors are counted elsewhere, this
  // CTA has nothing to do (block-uniform: every thread reads the same descriptors).
  auto elsewhere = [&](int c) {
    if ((tb->uniq_mask >> c) & 1u) return true;
    int64_t kmin, range;
    return A.agg && tb->agg[c] >= 0 && agg_active(A.agg[tb->agg[c]], tb->agg[c], A.ws, &kmin, &range);
  };
  const bool count_here = A.items == nullptr || tb->surv_by == kSurvRow;
  bool row_cols = false;
  for (int s = pair_begin / A.d; pair_end > pair_begin && s <= (pair_end - 1) / A.d && !row_cols; s++)
    if (!elsewhere(tb->key_col[s])) row_cols = true;
  if (!count_here && !row_cols) return;
  const int npairs = pair_end - pair_begin;
  const int w = A.w;
  const int64_t n_rows = tb->n_rows;
  const int filtered = tb->filtered;
  const bool vec = tb->vec_ok != 0;
  const int R = A.tile_rows;
  const int M = A.map_slots;

  // ---- shared memory carve-up
  // (region sizes must match build_smem_bytes)
  unsigned char* sp = smem;
  PairParam* prm = reinterpret_cast<PairParam*>(sp);
  sp += align16(sizeof(PairParam) * A.max_pairs);
  int32_t* plist = reinterpret_cast<int32_t*>(sp);  // slab pairs grouped by key column
  sp += align16(sizeof(int32_t) * A.max_pairs);
  int32_t* cnt = reinterpret_cast<int32_t*>(sp);  // private counters (mode 1)
  if (!GLOBAL) sp += align16(sizeof(int32_t) * size_t(A.smem_pairs) * w);
  unsigned long long* mkey = reinterpret_cast<unsigned long long*>(sp);
  if (DEDUPE) sp += align16(sizeof(unsigned long long) * size_t(M));
  int32_t* mcnt = reinterpret_cast<int32_t*>(sp);
  if (DEDUPE) sp += align16(sizeof(int32_t) * size_t(M));
  uint16_t* surv = reinterpret_cast<uint16_t*>(sp);
  sp += align16(sizeof(uint16_t) * R);
  int32_t* sint = reinterpret_cast<int32_t*>(sp);  // [0] tail, [1..32] warp sums, [39] #cols, [40..] columns
  int32_t* cols_list = sint + 40;                  // [CMP_MAX_COLS]
  int32_t* colstart = sint + 40 + CMP_MAX_COLS;    // [CMP_MAX_COLS + 1]

  for (int p = tid; p < npairs; p += T) {
    const int pair = pair_begin + p;
    const int s = pair / A.d, i = pair % A.d;
    const int e = tb->edge_id[s];
    prm[p] = make_pair_param(A.hash[size_t(e) * A.d + i]);
  }
  if (!GLOBAL)
    for (int j = tid; j < npairs * w; j += T) cnt[j] = 0;
  if (tid == 0) {
    // distinct key columns of the slab in first-use order, and the slab's pairs grouped
    // by column: plist[colstart[k] .. colstart[k+1]) are the pairs hashing column k
    int nc = 0;
    for (int p = 0; p < npairs; p++) {
      const int c = tb->key_col[(pair_begin + p) / A.d];
      bool seen = false;
      for (int q = 0; q < nc; q++) seen |= cols_list[q] == c;
      if (!seen) cols_list[nc++] = c;
    }
    int n = 0;
    for (int k = 0; k < nc; k++) {
      colstart[k] = n;
      for (int p = 0; p < npairs; p++)
        if (tb->key_col[(pair_begin + p) / A.d] == cols_list[k]) plist[n++] = p;
    }
    colstart[nc] = n;
    sint[39] = nc;
  }
  __syncthreads();
  const int n_keycols = sint[39];

  int32_t* gcnt = tb->counters + size_t(pair_begin) * w;
  int64_t my_survivors = 0;

  // Hash the first n_entries (field element, count) entries of mkey / mcnt for the pairs
  // of key column kc, or (no map) the keys of the tile's first n_entries survivors.  Two
  // entries per thread share every parameter load: two independent hash chains.
  auto hash_pairs = [&](auto smallx, const KeyPow& k0, const KeyPow& k1, int32_t m0, int32_t m1, int pl_begin,
                        int pl_end) {
    constexpr bool SMALLX = decltype(smallx)::value;
    for (int j = pl_begin; j < pl_end; j++) {
      const int pp = plist[j];
      const PairParam q = prm[pp];
      const uint32_t h0 = cw_bucket<POW2, SMALLX>(q, k0, uint32_t(w));
      const uint32_t h1 = cw_bucket<POW2, SMALLX>(q, k1, uint32_t(w));
      const int32_t v0 = cw_sign<SMALLX>(q, k0) * m0;
      const int32_t v1 = cw_sign<SMALLX>(q, k1) * m1;
      int32_t* row = (GLOBAL ? gcnt : cnt) + size_t(pp) * w;  // L2 counters, or the CTA's shared ones
      if (GLOBAL) {
        red_add(row + h0, v0);
        if (m1) red_add(row + h1, v1);
      } else {
        red_add_shared(row + h0, v0);
        if (m1) red_add_shared(row + h1, v1);
      }
    }
  };
  auto hash_entries = [&](int kc, int n_entries, const void* kbase, int32_t kdt, int64_t r0, bool from_map) {
    const int pl_begin = colstart[kc], pl_end = colstart[kc + 1];
    for (int e0 = tid; e0 < n_entries; e0 += 2 * T) {
      const int e1 = e0 + T;
      uint64_t x0, x1 = 0;
      int32_t m0, m1 = 0;
      if (from_map) {
        x0 = mkey[e0];
        m0 = mcnt[e0];
        if (e1 < n_entries) x1 = mkey[e1], m1 = mcnt[e1];
      } else {
        x0 = key_field(load1(kbase, kdt, r0 + (filtered ? surv[e0] : e0)));
        m0 = 1;
        if (e1 < n_entries) x1 = key_field(load1(kbase, kdt, r0 + (filtered ? surv[e1] : e1))), m1 = 1;
      }
      const KeyPow k0 = key_powers(x0);
      const KeyPow k1 = key_powers(x1);
      // keys below 2^31 (every non-negative int32 key) have a zero high limb
      if (__all_sync(__activemask(), (k0.x.hi | k1.x.hi) == 0))
        hash_pairs(std::true_type{}, k0, k1, m0, m1, pl_begin, pl_end);
      else
        hash_pairs(std::false_type{}, k0, k1, m0, m1, pl_begin, pl_end);
    }
  };

  {
    const int64_t n_tiles = (n_rows + R - 1) / R;
    for (int64_t tile = cta_in_slab; tile < n_tiles; tile += n_ctas) {
      const int64_t r0 = tile * R;
      const int rows_in_tile = int(min(int64_t(R), n_rows - r0));

      // ---------------- A. predicates and survivor compaction
      const int n_surv = tile_survivors(tb, r0, rows_in_tile, R, vec, surv, sint);
      if (count_here) my_survivors += n_surv;

      // ---------------- B. per key column: aggregate equal keys, hash, update
      for (int kc = 0; kc < n_keycols; kc++) {
        const int c = cols_list[kc];
        if (elsewhere(c)) continue;
        const void* kbase = tb->col[c];
        const int32_t kdt = tb->dtype[c];
        int n_entries = n_surv;
        // a tile with at most one survivor per thread is hashed directly: the map's clearing
        // and compaction would cost more than the duplicates it merges
        const bool use_map = DEDUPE && n_surv > T;  // block-uniform
        if (use_map) {
          for (int s = tid; s < M; s += T) {
            mkey[s] = kEmptyKey;
            mcnt[s] = 0;
          }
          __syncthreads();
          const uint32_t mmask = uint32_t(M - 1);
          for (int base = 0; base < n_surv; base += T) {  // block-uniform trip count
            const int e = base + tid;
            const bool valid = e < n_surv;
            unsigned long long x = kEmptyKey;
            if (valid) x = key_field(load1(kbase, kdt, r0 + (filtered ? surv[e] : e)));
            // equal keys of the warp are inserted once, by their lowest lane, with their count
            const unsigned peers = __match_any_sync(0xffffffffu, x);
            if (!valid || lane != __ffs(peers) - 1) continue;
            uint32_t slot = map_slot(x, mmask);
            bool done = false;
            for (int probe = 0; probe < M; probe++) {
              const unsigned long long prev = atomicCAS(&mkey[slot], kEmptyKey, x);
              if (prev == kEmptyKey || prev == x) {
                red_add_shared(&mcnt[slot], int32_t(__popc(peers)));
                done = true;
                break;
              }
              slot = (slot + 1) & mmask;
            }
            if (!done) set_status(A.status, CMP_ETIMEOUT);  // unreachable: M > tile rows
          }
          __syncthreads();
          // compact occupied slots to the front (read all, barrier, write all)
          const int spt = M / T;  // <= kMaxSlotsPerThread, host-checked
          unsigned long long kx[kMaxSlotsPerThread];
          int32_t kn[kMaxSlotsPerThread];
          uint32_t valid = 0;
#pragma unroll
          for (int j = 0; j < kMaxSlotsPerThread; j++) {
            kx[j] = kEmptyKey;
            kn[j] = 0;
            if (j < spt) {
              kx[j] = mkey[tid * spt + j];
              kn[j] = mcnt[tid * spt + j];
              if (kx[j] != kEmptyKey) valid |= 1u << j;
            }
          }
          const int mine = __popc(valid);
          int incl = mine;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
          }
          if (lane == 31) sint[1 + warp] = incl;
          __syncthreads();
          if (warp == 0) {
            const int nw = T >> 5;
            int v = lane < nw ? sint[1 + lane] : 0;
            int s2 = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int t = __shfl_up_sync(0xffffffffu, s2, o);
              if (lane >= o) s2 += t;
            }
            if (lane < nw) sint[1 + lane] = s2 - v;  // exclusive prefix per warp
            if (lane == nw - 1) sint[0] = s2;
          }
          __syncthreads();
          int pos = sint[1 + warp] + incl - mine;
          n_entries = sint[0];
#pragma unroll
          for (int j = 0; j < kMaxSlotsPerThread; j++) {
            if ((valid >> j) & 1u) {
              mkey[pos] = kx[j];
              mcnt[pos] = kn[j];
              pos++;
            }
          }
          __syncthreads();
        }
        hash_entries(kc, n_entries, kbase, kdt, r0, use_map);
        __syncthreads();  // map / survivor list reused next
      }
    }
  }

  // ---------------- C. flush private counters, count survivors once per table
  if (!GLOBAL) {
    __syncthreads();
    for (int j = tid; j < npairs * w; j += T) {
      const int32_t v = cnt[j];
      if (v) red_add(gcnt + j, v);
    }
  }
  if (pair_begin == 0 && tid == 0 && my_survivors)
    atomicAdd(reinterpret_cast<unsigned long long*>(tb->survivors), (unsigned long long)my_survivors);
}

size_t build_smem_bytes(const BuildShape& s, int w) {
  size_t b = align16(sizeof(PairParam) * s.max_pairs) + align16(sizeof(int32_t) * s.max_pairs);
  if (s.mode == 1) b += align16(sizeof(int32_t) * size_t(s.smem_pairs) * w);
  if (s.dedupe) b += align16(sizeof(unsigned long long) * size_t(s.map_slots)) + align16(sizeof(int32_t) * size_t(s.map_slots));
  b += align16(sizeof(uint16_t) * s.tile_rows);
  b += sizeof(int32_t) * (40 + 2 * CMP_MAX_COLS + 1);
  return b;
}

template <bool G, bool D, bool P>
static cudaError_t launch_one(const BuildArgs& a, const BuildShape& s, cudaStream_t st) {
  auto k = k_sketch_build<G, D, P>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem_bytes));
  if (e != cudaSuccess) return e;
  k<<<s.grid, s.threads, s.smem_bytes, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_build(const BuildArgs& a, const BuildShape& s, cudaStream_t st) {
  const bool pow2 = (a.w & (a.w - 1)) == 0;
  const bool g = s.mode == 2, d = s.dedupe != 0;
  if (g) {
    if (d) return pow2 ? launch_one<true, true, true>(a, s, st) : launch_one<true, true, false>(a, s, st);
    return pow2 ? launch_one<true, false, true>(a, s, st) : launch_one<true, false, false>(a, s, st);
  }
  if (d) return pow2 ? launch_one<false, true, true>(a, s, st) : launch_one<false, true, false>(a, s, st);
  return pow2 ? launch_one<false, false, true>(a, s, st) : launch_one<false, false, false>(a, s, st);
}

// ---------------------------------------------------------------- key aggregation
// Clears every aggregated column's count array (all cap slots: the surviving keys' range
// is only known after the counting pass); grid.y = column.  Arrays are 256-byte aligned
// and padded to whole int4 words.
__global__ void __launch_bounds__(256) k_agg_zero(const __grid_constant__ BuildArgs A) {
  const AggCol ac = A.agg[blockIdx.y];
  int4* c4 = reinterpret_cast<int4*>(A.ws + ac.off);
  // (a presence bitmap: its whole runs, then the int4 holding its PresenceCheck)
  const int64_t n4 = ac.kind == kAggPresence ? presence_words(ac.cap) / 4 + 1 : (ac.cap + 3) / 4;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x)
    c4[i] = make_int4(0, 0, 0, 0);
}

// survivor offsets: a tile's (generic path) or two 256-entry buffers per warp (warp path)
__host__ __device__ inline size_t agg_count_surv_entries(int32_t tile_rows, int32_t threads) {
  return tile_rows > 16 * threads ? size_t(tile_rows) : size_t(16) * threads;
}

// Counting pass of key aggregation.  Persistent CTAs take chunks of whole tiles of a
// table's rows (CountItem.chunk_rows) in order from an atomic counter.  For every surviving
// row and every aggregated key column of the table, the key's slot (key - base) & mask gets
// one count (a presence column: its bit is set; a bit found set already makes the column
// inactive): in the CTA's two-way set-associative shared-memory cache when a way of its set
// holds that slot index or is free (the frequent keys of a skewed column settle there),
// else with one global atomic on the count array.  Caches are added to the count arrays
// when the CTA moves to another table or ends.  The pass also records each column's
// smallest and largest surviving key (thread-local, then warp and CTA reductions, then one
// global atomic pair per column and table visit; a declared domain stands for them), and
// counts the table's survivors.
__global__ void __launch_bounds__(512, 2) k_agg_count(const __grid_constant__ BuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  // The unique-key kernel, launched next as a programmatic dependent, reads nothing this
  // pass writes: let it start now and share the SMs (this pass waits on memory, that one
  // on integer arithmetic).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ int32_t* acnt[CMP_MAX_SKETCHES];  // the current table's aggregated columns
  __shared__ int64_t abase[CMP_MAX_SKETCHES], acap[CMP_MAX_SKETCHES];
  __shared__ uint64_t amask[CMP_MAX_SKETCHES];
  __shared__ int32_t acol[CMP_MAX_SKETCHES], aidx[CMP_MAX_SKETCHES], akind[CMP_MAX_SKETCHES];
  __shared__ unsigned long long amax[CMP_MAX_SKETCHES], amin[CMP_MAX_SKETCHES];  // encoded
  __shared__ int32_t n_ac;
  __shared__ uint32_t akeys;  // the current table's aggregated key columns (bit c: column c)
  __shared__ long long next_chunk;
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
  const int R = A.tile_rows, H = A.cnt_cache_slots, n_cache = A.cnt_cache_cols;
  const int hshift = 32 - (31 - __clz(H));  // H is a power of two >= 256
  uint32_t* ckey = reinterpret_cast<uint32_t*>(smem);  // [n_cache][H] cached slot index
  uint32_t* ccnt = ckey + size_t(H) * n_cache;          // [n_cache][H] its count so far
  unsigned char* sp = smem + align16(sizeof(uint32_t) * 2 * size_t(H) * n_cache);
  uint16_t* surv = reinterpret_cast<uint16_t*>(sp);
  sp += align16(sizeof(uint16_t) * agg_count_surv_entries(R, T));
  int32_t* sint = reinterpret_cast<int32_t*>(sp);
  constexpr uint32_t kEmpty = 0xFFFFFFFFu;  // never a slot index: cap <= 2^31 - 1
  // this launch's chunk counter: slot 0 (the only launch, or the first of two), 2 (the second)
  unsigned long long* work = reinterpret_cast<unsigned long long*>(A.ws) + 2 * int64_t(A.n_agg) + A.cnt_work_slot;

  // One surviving key of column a.  Returns false when the key lies outside the column's
  // declared domain (its counts are then discarded: the column keeps the per-row path).
  // The hot-key cache of one column: H / 2 sets of two (key, count) slots, a set chosen by a
  // multiplicative hash of the slot index x.  x is counted in the way that holds it, else in
  // an empty way it claims (compare-and-swap; a way once claimed keeps its key until the
  // flush), else not at all (returns false: the caller counts it in the global array).
  auto cache_count = [&](uint32_t* keys, uint32_t* cnts, uint32_t x) {
    const uint32_t set2 = ((x * 0x9E3779B1u) >> (hshift + 1)) * 2;
    const unsigned long long both = *reinterpret_cast<volatile unsigned long long*>(keys + set2);
    const uint2 cur = make_uint2(uint32_t(both), uint32_t(both >> 32));
    if (cur.x == x || cur.y == x) {
      red_add_shared(cnts + set2 + (cur.x == x ? 0 : 1), 1u);
      return true;
    }
    for (int way = cur.x == kEmpty ? 0 : (cur.y == kEmpty ? 1 : 2); way < 2; way++) {
      const uint32_t prev = atomicCAS(keys + set2 + way, kEmpty, x);
      if (prev == kEmpty || prev == x) {
        red_add_shared(cnts + set2 + way, 1u);
        return true;
      }
    }
    return false;
  };
  auto count_key = [&](int a, int64_t key) {
    const uint64_t off = uint64_t(key) - uint64_t(abase[a]);
    if (amask[a] == ~0ull && off >= uint64_t(acap[a])) return false;
    if (akind[a] == kAggPresence) {  // off < cap <= 2^32; repeated keys are found by k_presence_check
      red_or(reinterpret_cast<uint32_t*>(acnt[a]) + (off >> 5), 1u << (off & 31));
      return true;
    }
    const uint32_t x = uint32_t(off & amask[a]);  // < cap
    if (a < n_cache && cache_count(ckey + size_t(a) * H, ccnt + size_t(a) * H, x)) return true;
    red_add(acnt[a] + x, 1);
    return true;
  };
  // thread-local key range of column a -> shared (warp-reduced first)
  auto fold_range = [&](int a, int64_t mn, int64_t mx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mn, o));
      mx = max(mx, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mx, o));
    }
    if (lane == 0 && mx >= mn) {
      atomicMax(&amax[a], (unsigned long long)enc_max(mx));
      atomicMax(&amin[a], (unsigned long long)enc_min(mn));
    }
  };
  // A counted column's parameters in registers (warp path).
  struct CntCol {
    int32_t* cnt;
    uint32_t* ckey;  // its cache (nullptr: not cached)
    uint32_t* ccnt;
    uint64_t base, cap, mask;
    bool declared;
  };
  auto cnt_col = [&](int a) {
    CntCol cc;
    cc.cnt = acnt[a];
    cc.ckey = a < n_cache ? ckey + size_t(a) * H : nullptr;
    cc.ccnt = a < n_cache ? ccnt + size_t(a) * H : nullptr;
    cc.base = uint64_t(abase[a]);
    cc.cap = uint64_t(acap[a]);
    cc.mask = amask[a];
    cc.declared = amask[a] == ~0ull;
    return cc;
  };
  // adds the caches and key ranges of the current table to the global arrays (block-wide)
  auto flush = [&]() {
    __syncthreads();
    for (int a = 0; a < min(int(n_ac), n_cache); a++)
      for (int s = tid; s < H; s += T) {
        const uint32_t k = ckey[size_t(a) * H + s];
        if (k != kEmpty) red_add(acnt[a] + k, int32_t(ccnt[size_t(a) * H + s]));
      }
    if (tid < n_ac && amax[tid] != 0) {
      unsigned long long* st = reinterpret_cast<unsigned long long*>(A.ws) + 2 * int64_t(aidx[tid]);
      atomicMax(st, amax[tid]);
      atomicMax(st + 1, amin[tid]);
    }
    __syncthreads();
  };

  // the item of chunk c (items are in chunk order)
  auto item_of = [&](int64_t c) {
    int it = 0;
    while (it + 1 < A.n_cnt_items && A.cnt_items[it + 1].chunk_begin <= c) it++;
    return it;
  };
  // Memory-level parallelism: each warp prefetches into L2 the rows it reads next (bulk
  // prefetches of whole row ranges, or the key sectors of its survivors): no registers or
  // shared memory are held for data in flight.
  int item = -1;  // block-uniform
  for (;;) {
    if (tid == 0) next_chunk = A.cnt_chunk_begin + (long long)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t c = next_chunk;
    if (c >= A.cnt_chunk_end) break;  // block-uniform
    const int it = item_of(c);
    const CountItem ci = A.cnt_items[it];
    const DevTable* tb = A.tables + ci.table;
    if (it != item) {  // a new table: flush the caches, then set them up for its columns
      if (item >= 0) flush();
      if (tid == 0) {
        int n = 0;
        uint32_t keys = 0;
        for (int col = 0; col < tb->n_cols; col++)
          if (tb->agg[col] >= 0) keys |= 1u << col;
        akeys = keys;
        // count arrays first (they take the hot-key caches), then presence bitmaps
        for (int kind = kAggCount; kind <= kAggPresence; kind++)
          for (int col = 0; col < tb->n_cols && n < CMP_MAX_SKETCHES; col++) {
            const int ai = tb->agg[col];
            if (ai < 0 || A.agg[ai].kind != kind) continue;
            const AggCol& ac = A.agg[ai];
            acnt[n] = reinterpret_cast<int32_t*>(A.ws + ac.off);
            abase[n] = ac.base;
            acap[n] = ac.cap;
            amask[n] = ac.mask;
            acol[n] = col;
            aidx[n] = ai;
            akind[n] = kind;
            amax[n] = 0;
            amin[n] = 0;
            n++;
          }
        n_ac = n;
      }
      for (int s = tid; s < H * n_cache; s += T) {
        ckey[s] = kEmpty;
        ccnt[s] = 0;
      }
      item = it;
      __syncthreads();
    }
    const int nac = n_ac;
    const int64_t n_rows = tb->n_rows;
    const int64_t r_begin = (c - ci.chunk_begin) * ci.chunk_rows, r_end = min(n_rows, r_begin + ci.chunk_rows);
    const bool vec = tb->vec_ok != 0;
    if (!tb->filtered) {
      if (tid == 0 && r_end > r_begin)
        atomicAdd(reinterpret_cast<unsigned long long*>(tb->survivors), (unsigned long long)(r_end - r_begin));
      // every row survives: eight consecutive rows per thread and step, two 16-byte loads
      // for int32 keys
      for (int a = 0; a < nac; a++) {
        const void* kbase = tb->col[acol[a]];
        const int32_t kdt = tb->dtype[acol[a]];
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        bool ok = true;
        for (int64_t r = r_begin + 8 * int64_t(tid); r < r_end; r += 8 * int64_t(T)) {
          if (lane == 0) {  // this warp's 256 rows of the next step (this column, else the next one's first)
            const int64_t rw = r + 8 * int64_t(T);
            if (rw < r_end) {
              prefetch_rows(tb, 1u << acol[a], rw, min(r_end, rw + 256), 0, 1);
            } else if (a + 1 < nac) {
              const int64_t rn = r_begin + (rw - r_begin) % (8 * int64_t(T));
              prefetch_rows(tb, 1u << acol[a + 1], rn, min(r_end, rn + 256), 0, 1);
            }
          }
          int64_t v[8];
          int nv = int(min(int64_t(8), r_end - r));
          if (vec && nv == 8) {
            if (kdt == CMP_I32) {
              const int4* p = reinterpret_cast<const int4*>(reinterpret_cast<const int32_t*>(kbase) + r);
              const int4 u = __ldg(p), q = __ldg(p + 1);
              v[0] = u.x, v[1] = u.y, v[2] = u.z, v[3] = u.w, v[4] = q.x, v[5] = q.y, v[6] = q.z, v[7] = q.w;
            } else {
              const longlong2* p = reinterpret_cast<const longlong2*>(reinterpret_cast<const long long*>(kbase) + r);
#pragma unroll
              for (int h = 0; h < 4; h++) {
                const longlong2 u = __ldg(p + h);
                v[2 * h] = u.x, v[2 * h + 1] = u.y;
              }
            }
          } else {
            for (int q = 0; q < 8; q++) v[q] = q < nv ? load1(kbase, kdt, r + q) : 0;
          }
#pragma unroll
          for (int q = 0; q < 8; q++)
            if (q < nv) {
              mn = min(mn, v[q]);
              mx = max(mx, v[q]);
              ok &= count_key(a, v[q]);
            }
        }
        if (!ok) mn = INT64_MIN, mx = INT64_MAX;  // outside the declared domain: out of range
        fold_range(a, mn, mx);
      }
    } else if (vec && !tb->sample_keep && tb->n_preds >= 1 && tb->n_preds <= 2 && nac <= 2 &&
               tb->dtype[tb->pred[0].col] == CMP_I32 && tb->dtype[tb->pred[tb->n_preds - 1].col] == CMP_I32 &&
               akind[0] == kAggCount && akind[nac - 1] == kAggCount) {
      // Warp-autonomous scan in three stages (no block barrier inside the chunk).  Warp w
      // takes the 256-row steps w, w + nwarps, ...; lane l the 16-byte groups at 4 l and 128 +
      // 4 l of a step.  While it counts the survivors of step s (lane e holds the keys of
      // survivor e, loaded during step s - 1), the predicate loads of step s + 1 (prefetched
      // into L2 during step s - 1) are in flight; then it compacts step s + 1's survivors
      // into its other 256-entry buffer and issues the loads of their keys, and bulk-
      // prefetches the predicate rows of step s + 2.  Only the key sectors holding survivors
      // are read.
      const int warp = tid >> 5, nwarps = T >> 5;
      uint16_t* wb0 = surv + warp * 512;  // two 256-entry buffers: wb0 + 256 * buf
      const PredReg q0 = pred_reg(tb->pred[0]);  // in registers for the whole chunk
      const PredReg q1 = pred_reg(tb->pred[tb->n_preds - 1]);
      const int32_t* c0 = reinterpret_cast<const int32_t*>(tb->col[tb->pred[0].col]);
      const int32_t* c1 = reinterpret_cast<const int32_t*>(tb->col[tb->pred[tb->n_preds - 1].col]);
      const void* kb0 = tb->col[acol[0]];
      const void* kb1 = nac > 1 ? tb->col[acol[1]] : kb0;
      const int32_t kd0 = tb->dtype[acol[0]], kd1 = nac > 1 ? tb->dtype[acol[1]] : kd0;
      int64_t mn0 = INT64_MAX, mx0 = INT64_MIN, mn1 = INT64_MAX, mx1 = INT64_MIN;
      bool ok0 = true, ok1 = true;
      unsigned long long n_surv = 0;
      const CntCol cc0 = cnt_col(0), cc1 = cnt_col(nac > 1 ? 1 : 0);
      // A cache miss is counted with a global atomic one step later (at most one per lane and
      // column; a second one in the same step at once), its count-array line prefetched into
      // L2 now: the atomic then finds the line in L2 instead of waiting for DRAM there.
      uint32_t pend0 = kEmpty, pend1 = kEmpty;
      auto count_deferred = [&](const CntCol& cc, int64_t key, uint32_t& pend) {
        const uint64_t off = uint64_t(key) - cc.base;
        if (cc.declared && off >= cc.cap) return false;
        const uint32_t x = uint32_t(off & cc.mask);
        if (cc.ckey && cache_count(cc.ckey, cc.ccnt, x)) return true;
        if (pend == kEmpty) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(cc.cnt + x)));
          pend = x;
        } else {
          red_add(cc.cnt + x, 1);
        }
        return true;
      };
      const int64_t stride = int64_t(nwarps) * 256;
      const int64_t rb_first = r_begin + int64_t(warp) * 256;
      // bulk L2 prefetch of the predicate rows of the step at rb (lanes 0 and 1)
      // (rb is a multiple of 4 rows from the 16-byte aligned columns: a whole step is one
      // aligned 1 KB prefetch per column; a partial last step is not prefetched)
      auto prefetch_preds = [&](int64_t rb) {
        if (lane < 2 && rb + 256 <= r_end) l2_prefetch_exact((lane == 0 ? c0 : c1) + rb, 1024u);
      };
      int4 v0[2], v1[2];  // predicate values of the next step: groups 4 l and 128 + 4 l
      int64_t pk0 = 0, pk1 = 0;  // keys of this lane's first survivor of the next step
      int nv[2];
      auto load_preds = [&](int64_t rb) {
        if (rb + 256 <= r_end) {  // a whole step (warp-uniform): no bounds per group
#pragma unroll
          for (int g = 0; g < 2; g++) {
            const int64_t r = rb + 128 * g + 4 * lane;
            nv[g] = 4;
            v0[g] = __ldg(reinterpret_cast<const int4*>(c0 + r));
            v1[g] = __ldg(reinterpret_cast<const int4*>(c1 + r));
          }
          return;
        }
#pragma unroll
        for (int g = 0; g < 2; g++) {
          const int64_t r = rb + 128 * g + 4 * lane;
          nv[g] = int(max(int64_t(0), min(int64_t(4), r_end - r)));
          if (nv[g] == 4) {
            v0[g] = __ldg(reinterpret_cast<const int4*>(c0 + r));
            v1[g] = __ldg(reinterpret_cast<const int4*>(c1 + r));
          } else {
            int t0[4], t1[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
              t0[j] = j < nv[g] ? __ldg(c0 + r + j) : 0;
              t1[j] = j < nv[g] ? __ldg(c1 + r + j) : 0;
            }
            v0[g] = make_int4(t0[0], t0[1], t0[2], t0[3]);
            v1[g] = make_int4(t1[0], t1[1], t1[2], t1[3]);
          }
        }
      };
      // the survivors of the step at rb (predicates in v0, v1) into buffer wbuf; their key
      // sectors are prefetched into L2.  Returns the count (warp-uniform).
      const bool ranges = !q0.in && !q1.in;  // the common case: two range / point predicates
      const PredI32 p0 = pred_i32(tb->pred[0]), p1 = pred_i32(tb->pred[tb->n_preds - 1]);
      auto compact = [&](int64_t rb, uint16_t* wbuf) {
        uint32_t m = 0;
#pragma unroll
        for (int g = 0; g < 2; g++) {
          const int a0[4] = {v0[g].x, v0[g].y, v0[g].z, v0[g].w}, a1[4] = {v1[g].x, v1[g].y, v1[g].z, v1[g].w};
          if (ranges) {
#pragma unroll
            for (int j = 0; j < 4; j++)
              m |= uint32_t(j < nv[g] && i32_holds(p0, a0[j]) && i32_holds(p1, a1[j])) << (4 * g + j);
          } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
              if (j < nv[g] && reg_holds(q0, a0[j]) && reg_holds(q1, a1[j])) m |= 1u << (4 * g + j);
          }
        }
        const int c = __popc(m);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int pos = incl - c;
        while (m) {  // this lane's survivors, in row order
          const int b = __ffs(m) - 1;
          m &= m - 1;
          wbuf[pos++] = uint16_t(128 * (b >> 2) + 4 * lane + (b & 3));
        }
        __syncwarp();
        if (lane < total) {  // the keys of survivor `lane`, loaded now and counted next step
          const int64_t row = rb + wbuf[lane];
          pk0 = load1(kb0, kd0, row);
          if (nac > 1) pk1 = load1(kb1, kd1, row);
        }
        return total;
      };
      // prologue: predicates of steps 0 and 1 prefetched, step 0 compacted
      prefetch_preds(rb_first);
      prefetch_preds(rb_first + stride);
      int n_cur = 0;
      if (rb_first < r_end) {
        load_preds(rb_first);
        n_cur = compact(rb_first, wb0);
      }
      int buf = 0;
      for (int64_t rb = rb_first; rb < r_end; rb += stride) {  // warp-uniform
        const int64_t rn = rb + stride;
        prefetch_preds(rn + stride);
        if (rn < r_end) load_preds(rn);  // in flight while step rb is counted
        n_surv += unsigned(n_cur);
        const uint16_t* cur = wb0 + 256 * buf;
        // the global atomics of last step's cache misses: their lines were prefetched then
        if (pend0 != kEmpty) red_add(cc0.cnt + pend0, 1);
        if (pend1 != kEmpty) red_add(cc1.cnt + pend1, 1);
        pend0 = pend1 = kEmpty;
        auto count_row = [&](int64_t k0, int64_t k1) {
          if (!cc0.declared) mn0 = min(mn0, k0), mx0 = max(mx0, k0);
          ok0 &= count_deferred(cc0, k0, pend0);
          if (nac > 1) {
            if (!cc1.declared) mn1 = min(mn1, k1), mx1 = max(mx1, k1);
            ok1 &= count_deferred(cc1, k1, pend1);
          }
        };
        if (lane < n_cur) count_row(pk0, pk1);
        for (int e = lane + 32; e < n_cur; e += 32) {  // beyond 32 survivors: loaded here
          const int64_t row = rb + cur[e];
          count_row(load1(kb0, kd0, row), nac > 1 ? load1(kb1, kd1, row) : 0);
        }
        __syncwarp();
        buf ^= 1;
        n_cur = rn < r_end ? compact(rn, wb0 + 256 * buf) : 0;
      }
      if (pend0 != kEmpty) red_add(cc0.cnt + pend0, 1);
      if (pend1 != kEmpty) red_add(cc1.cnt + pend1, 1);
      if (lane == 0 && n_surv) atomicAdd(reinterpret_cast<unsigned long long*>(tb->survivors), n_surv);
      // a declared domain holds every surviving key unless one left it: its range is the domain
      if (cc0.declared) mn0 = int64_t(cc0.base), mx0 = int64_t(cc0.base + cc0.cap - 1);
      if (!ok0) mn0 = INT64_MIN, mx0 = INT64_MAX;
      fold_range(0, mn0, mx0);
      if (nac > 1) {
        if (cc1.declared) mn1 = int64_t(cc1.base), mx1 = int64_t(cc1.base + cc1.cap - 1);
        if (!ok1) mn1 = INT64_MIN, mx1 = INT64_MAX;
        fold_range(1, mn1, mx1);
      }
    } else {
      for (int64_t r0 = r_begin; r0 < r_end; r0 += R) {
        if (tid < 32 && r0 + R < r_end) prefetch_rows(tb, akeys, r0 + R, min(r_end, r0 + 2 * int64_t(R)), tid, 32);
        const int rows_in_tile = int(min(int64_t(R), r_end - r0));
        const int n_surv = tile_survivors(tb, r0, rows_in_tile, R, vec, surv, sint);
        if (tid == 0 && n_surv)
          atomicAdd(reinterpret_cast<unsigned long long*>(tb->survivors), (unsigned long long)n_surv);
        for (int a = 0; a < nac; a++) {
          const void* kbase = tb->col[acol[a]];
          const int32_t kdt = tb->dtype[acol[a]];
          int64_t mn = INT64_MAX, mx = INT64_MIN;
          bool ok = true;
          for (int e = tid; e < n_surv; e += T) {
            const int64_t k = load1(kbase, kdt, r0 + surv[e]);
            mn = min(mn, k);
            mx = max(mx, k);
            ok &= count_key(a, k);
          }
          if (!ok) mn = INT64_MIN, mx = INT64_MAX;  // outside the declared domain: out of range
          fold_range(a, mn, mx);
        }
        __syncthreads();  // surv is rewritten by the next tile
      }
    }
    __syncthreads();  // next_chunk is rewritten next
  }
  if (item >= 0) flush();
}

// Hashing of the aggregated key columns: every nonzero (key, count) entry of a count array
// is hashed once per (sketch, row) pair on that column, and count * xi is added to the
// global counters.  Persistent CTAs take chunks of count-array slots in order from an
// atomic counter; a CTA loads the pairs' parameters when its column changes.  Each warp
// compacts the nonzero entries of its part of a chunk, 32 slots at a time, into a 96-entry
// buffer and hashes 64 of them, two per lane, whenever it holds 64.
constexpr int kHashThreads = 512;

constexpr int kHashPer = 2;                    // entries per lane and batch: independent hash chains
constexpr int kHashBatch = 32 * kHashPer;        // entries hashed at a time by a warp
constexpr int kHashBuf = kHashBatch + 32;        // entries buffered per warp (31 carried over)

size_t agg_hash_smem_bytes(int32_t max_pairs) {
  return align16(sizeof(PairParam) * size_t(max_pairs)) + align16(sizeof(int32_t*) * size_t(max_pairs)) +
         (kHashThreads / 32) * kHashBuf * (sizeof(unsigned long long) + sizeof(int32_t));
}

template <bool POW2>
__global__ void __launch_bounds__(kHashThreads) k_agg_hash(const __grid_constant__ BuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  // the presence-bitmap kernel, launched next as a programmatic dependent, reads nothing
  // this pass writes: let it start now
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ long long next_chunk;
  __shared__ int32_t n_pairs, active;
  __shared__ long long s_kmin, s_range;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int mp = A.hash_max_pairs;
  PairParam* prm = reinterpret_cast<PairParam*>(smem);
  int32_t** prow = reinterpret_cast<int32_t**>(smem + align16(sizeof(PairParam) * size_t(mp)));
  unsigned long long* bkey = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(prow) +
                                                                   align16(sizeof(int32_t*) * size_t(mp))) +
                             kHashBuf * warp;
  int32_t* bcnt = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned long long*>(
                      reinterpret_cast<unsigned char*>(prow) + align16(sizeof(int32_t*) * size_t(mp))) +
                                             kHashBuf * nw) +
                  kHashBuf * warp;
  unsigned long long* work = reinterpret_cast<unsigned long long*>(A.ws) + 2 * int64_t(A.n_agg) + 1;
  const uint32_t w = uint32_t(A.w);
  int cur = -1;  // block-uniform
  for (;;) {
    if (tid == 0) next_chunk = (long long)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t c = next_chunk;
    if (c >= A.hash_total_chunks) break;
    int ai = 0;
    while (ai + 1 < A.n_agg && A.agg[ai + 1].hash_chunk0 <= c) ai++;
    const AggCol ac = A.agg[ai];
    const DevTable* tb = A.tables + ac.table;
    if (ai != cur) {  // a new column: its pairs' parameters and counter rows
      if (tid == 0) {
        int64_t kmin = 0, range = 0;
        active = agg_active(ac, ai, A.ws, &kmin, &range) ? 1 : 0;
        s_kmin = kmin;
        s_range = range;
        int n = 0;
        for (int s = 0; s < tb->n_sketches; s++)
          if (tb->key_col[s] == ac.col) n += A.d;
        n_pairs = n;
      }
      __syncthreads();
      const int np = n_pairs;
      for (int p = tid; p < np; p += blockDim.x) {
        int s = 0, k = p / A.d;  // the k-th sketch on this column
        for (;; s++)
          if (tb->key_col[s] == ac.col && k-- == 0) break;
        const int i = p % A.d;
        prm[p] = make_pair_param(A.hash[size_t(tb->edge_id[s]) * A.d + i]);
        prow[p] = tb->counters + (size_t(s) * A.d + i) * w;
      }
      cur = ai;
      __syncthreads();
    }
    const int64_t s0 = (c - ac.hash_chunk0) * kHashChunk, range = s_range;
    if (active && s0 < range) {
      const int32_t* cnts = reinterpret_cast<const int32_t*>(A.ws + ac.off);
      const int64_t kmin = s_kmin;
      // key kmin + j sits in slot (kmin - base + j) & mask
      const uint64_t off0 = uint64_t(kmin) - uint64_t(ac.base), mask = ac.mask;
      const int np = n_pairs;
      const int64_t per = kHashChunk / nw;  // a multiple of 32
      const int64_t ws0 = min(range, s0 + warp * per), ws1 = min(range, ws0 + per);
      // the first n entries of the warp's buffer, lane l taking l, l + 32, ...: kHashPer
      // independent hash chains per lane sharing every parameter load
      auto hash_batch = [&](int n) {
        KeyPow k[kHashPer];
        int32_t m[kHashPer];
        uint32_t hi_or = 0;
#pragma unroll
        for (int e = 0; e < kHashPer; e++) {
          const int j = lane + 32 * e;
          m[e] = j < n ? bcnt[j] : 0;
          k[e] = key_powers(j < n ? bkey[j] : 0);
          hi_or |= k[e].x.hi;
        }
        auto run = [&](auto smallx) {
          constexpr bool SX = decltype(smallx)::value;
          for (int p = 0; p < np; p++) {
            const PairParam q = prm[p];
            int32_t* row = prow[p];
#pragma unroll
            for (int e = 0; e < kHashPer; e++) {
              const uint32_t h = cw_bucket<POW2, SX>(q, k[e], w);
              const int32_t v = cw_sign<SX>(q, k[e]) * m[e];
              if (m[e]) red_add(row + h, v);
            }
          }
        };
        if (__all_sync(0xffffffffu, hi_or == 0)) run(std::true_type{});
        else run(std::false_type{});
      };
      int nb = 0;  // warp-uniform
      for (int64_t sb = ws0; sb < ws1; sb += 32) {
        const int64_t j = sb + lane;
        const int32_t cnt = j < ws1 ? __ldg(cnts + ((off0 + uint64_t(j)) & mask)) : 0;
        const unsigned nz = __ballot_sync(0xffffffffu, cnt != 0);
        if (cnt != 0) {
          const int pos = nb + __popc(nz & ((1u << lane) - 1u));
          bkey[pos] = key_field(kmin + j);
          bcnt[pos] = cnt;
        }
        nb += __popc(nz);
        __syncwarp();
        if (nb >= kHashBatch) {
          hash_batch(kHashBatch);
          __syncwarp();
          if (lane < nb - kHashBatch) {  // keep the overflow at the front
            bkey[lane] = bkey[kHashBatch + lane];
            bcnt[lane] = bcnt[kHashBatch + lane];
          }
          nb -= kHashBatch;
          __syncwarp();
        }
      }
      if (nb > 0) hash_batch(nb);
    }
    __syncthreads();  // next_chunk and the parameters are rewritten next
  }
}

cudaError_t launch_agg_hash(const BuildArgs& a, int32_t grid, cudaStream_t st) {
  if (a.n_agg <= 0 || grid <= 0) return cudaSuccess;
  const size_t smem = agg_hash_smem_bytes(a.hash_max_pairs);
  const bool pow2 = (a.w & (a.w - 1)) == 0;
  cudaError_t e = pow2 ? cudaFuncSetAttribute(k_agg_hash<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))
                       : cudaFuncSetAttribute(k_agg_hash<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  if (pow2) k_agg_hash<true><<<unsigned(grid), kHashThreads, smem, st>>>(a);
  else k_agg_hash<false><<<unsigned(grid), kHashThreads, smem, st>>>(a);
  return cudaGetLastError();
}

size_t agg_count_smem_bytes(int32_t tile_rows, int32_t cache_slots, int32_t cache_cols, int32_t threads) {
  return align16(sizeof(uint32_t) * 2 * size_t(cache_slots) * size_t(cache_cols)) +
         align16(sizeof(uint16_t) * agg_count_surv_entries(tile_rows, threads)) + sizeof(int32_t) * 40;
}

// After the counting pass: a presence column is valid only if its bitmap holds as many set
// bits as its table has rows (the table has no predicates: every row survives); fewer bits
// mean a key was seen twice, and the column's key range is then set to the whole int64
// range, so that agg_active turns it down.  Each CTA adds the set bits of its part of the
// bitmap; the CTA that finishes last (ticket) compares.  Grid: (CTAs per column, columns).
__global__ void __launch_bounds__(256) k_presence_check(const __grid_constant__ BuildArgs A) {
  __shared__ unsigned long long part[8];
  __shared__ bool last;
  const AggCol ac = A.agg[blockIdx.y];
  if (ac.kind != kAggPresence) return;  // block-uniform
  const int64_t words = presence_words(ac.cap);
  const uint32_t* bm = reinterpret_cast<const uint32_t*>(A.ws + ac.off);
  PresenceCheck* pc = reinterpret_cast<PresenceCheck*>(A.ws + ac.off + 4 * words);
  unsigned long long n = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < words; i += int64_t(gridDim.x) * blockDim.x)
    n += __popc(__ldg(bm + i));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int wi = 0; wi < int(blockDim.x >> 5); wi++) t += part[wi];
    atomicAdd(&pc->bits, t);
    __threadfence();  // this CTA's total before its ticket
    last = atomicAdd(&pc->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  const unsigned long long total = *reinterpret_cast<volatile unsigned long long*>(&pc->bits);
  if (total != (unsigned long long)A.tables[ac.table].n_rows) {
    unsigned long long* st = reinterpret_cast<unsigned long long*>(A.ws) + 2 * int64_t(blockIdx.y);
    atomicMax(st, (unsigned long long)enc_max(INT64_MAX));
    atomicMax(st + 1, (unsigned long long)enc_min(INT64_MIN));
  }
}

cudaError_t launch_presence_check(const BuildArgs& a, cudaStream_t st) {
  if (a.n_agg <= 0 || a.n_ditems <= 0) return cudaSuccess;
  k_presence_check<<<dim3(unsigned(std::max(1, sm_count())), unsigned(a.n_agg)), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_agg_zero(const BuildArgs& a, cudaStream_t st) {
  if (a.n_agg <= 0) return cudaSuccess;
  const dim3 g(unsigned(std::max(1, 8 * sm_count() / std::max(1, a.n_agg))), unsigned(a.n_agg));
  k_agg_zero<<<g, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// One launch of the counting pass over chunks [chunk_begin, chunk_end), taken from chunk
// counter `work_slot` of the workspace header (zeroed before the build).
cudaError_t launch_agg_count(const BuildArgs& a, int32_t tile_rows, int32_t cnt_threads, int32_t cnt_grid,
                             int32_t work_slot, int64_t chunk_begin, int64_t chunk_end, cudaStream_t st) {
  if (a.n_agg <= 0 || cnt_grid <= 0 || chunk_end <= chunk_begin) return cudaSuccess;
  const size_t smem = agg_count_smem_bytes(tile_rows, a.cnt_cache_slots, a.cnt_cache_cols, cnt_threads);
  cudaError_t e = cudaFuncSetAttribute(k_agg_count, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  // the whole shared memory of the SM, so that a CTA of the unique-key or the dense kernel
  // (launched next, as a programmatic dependent) fits beside one of this pass
  e = cudaFuncSetAttribute(k_agg_count, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  BuildArgs b = a;
  b.cnt_work_slot = work_slot;
  b.cnt_chunk_begin = chunk_begin;
  b.cnt_chunk_end = chunk_end;
  k_agg_count<<<unsigned(cnt_grid), cnt_threads, smem, st>>>(b);
  return cudaGetLastError();
}

__global__ void k_zero_spans(const ZeroSpan* __restrict__ spans, int32_t n) {
  // one block-stride pass per span; spans are 4-byte multiples: 4-byte stores up to the
  // first 16-byte boundary, 16-byte stores, then 4-byte stores for the tail
  for (int32_t s = blockIdx.y; s < n; s += gridDim.y) {
    const ZeroSpan z = spans[s];
    uint32_t* p = reinterpret_cast<uint32_t*>(z.ptr);
    const int64_t words = z.bytes / 4;
    const int64_t head = min(words, int64_t((16 - (reinterpret_cast<uintptr_t>(p) & 15)) & 15) / 4);
    const int64_t n4 = (words - head) / 4;
    const int64_t i0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, step = int64_t(gridDim.x) * blockDim.x;
    if (i0 < head) p[i0] = 0;
    int4* q = reinterpret_cast<int4*>(p + head);
    for (int64_t i = i0; i < n4; i += step) q[i] = make_int4(0, 0, 0, 0);
    for (int64_t i = head + 4 * n4 + i0; i < words; i += step) p[i] = 0;
  }
}

cudaError_t launch_zero_spans(const ZeroSpan* spans_dev, int32_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(64, unsigned(n < 1024 ? n : 1024));
  k_zero_spans<<<grid, 256, 0, st>>>(spans_dev, n);
  return cudaGetLastError();
}

}  // namespace cmpk
