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
// Key aggregation (batched build, large tables): before the build kernel, k_agg_stats
// finds each aggregated key column's smallest and largest key, k_agg_zero clears the
// used part of its count array, and k_agg_count adds every tile's survivors to it (tile
// keys reduced in a shared-memory map first, one global atomic per distinct key of the
// tile).  The build kernel's aggregated items then hash each nonzero (key, count) entry
// once per pair instead of once per tuple, and its row items skip those columns.
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
  int pair_begin, pair_end, cta_in_slab, n_ctas, agg_item = -1;
  if (A.items) {
    const BuildItem it = A.items[A.cta_item[blockIdx.x]];
    tb = A.tables + it.table;
    pair_begin = it.pair_begin;
    pair_end = it.pair_end;
    cta_in_slab = int(blockIdx.x) - it.first_cta;
    n_ctas = it.n_ctas;
    agg_item = it.agg;
  } else {
    tb = &A.table;
    const int slab = int(blockIdx.x) / A.ctas_per_slab;
    cta_in_slab = int(blockIdx.x) % A.ctas_per_slab;
    n_ctas = A.ctas_per_slab;
    pair_begin = slab * A.pairs_per_slab;
    const int total_pairs = tb->n_sketches * A.d;
    pair_end = min(pair_begin + A.pairs_per_slab, total_pairs);
  }
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
      int32_t* row = (GLOBAL ? gcnt : cnt) + size_t(pp) * w;
      atomicAdd(row + h0, v0);
      if (m1) atomicAdd(row + h1, v1);
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

  if (agg_item >= 0) {
    // ---------------- aggregated column: chunks of its count array
    if constexpr (DEDUPE) {
      const AggCol ac = A.agg[agg_item];
      int64_t kmin = 0, range = 0;
      int kc = -1;
      for (int k = 0; k < n_keycols; k++)
        if (cols_list[k] == ac.col) kc = k;
      if (kc >= 0 && agg_active(ac, agg_item, A.ws, &kmin, &range)) {
        const int32_t* cnts = reinterpret_cast<const int32_t*>(A.ws + ac.off);
        const int64_t n_chunks = (range + M - 1) / M;  // chunks of the entry lists' capacity
        for (int64_t chunk = cta_in_slab; chunk < n_chunks; chunk += n_ctas) {
          const int64_t i0 = chunk * M;
          const int nin = int(min(int64_t(M), range - i0));
          if (tid == 0) sint[0] = 0;
          __syncthreads();
          for (int base = 0; base < nin; base += T) {  // block-uniform trip count
            const int j = base + tid;
            const int32_t c = j < nin ? __ldg(cnts + i0 + j) : 0;
            const unsigned nz = __ballot_sync(0xffffffffu, c != 0);
            int wbase = 0;
            if (lane == 0 && nz) wbase = atomicAdd(&sint[0], __popc(nz));
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            if (c != 0) {
              const int pos = wbase + __popc(nz & ((1u << lane) - 1u));
              mkey[pos] = key_field(kmin + i0 + j);
              mcnt[pos] = c;
            }
          }
          __syncthreads();
          hash_entries(kc, sint[0], nullptr, 0, 0, true);
          __syncthreads();  // entry lists reused next
        }
      }
    }
  } else {
    const int64_t n_tiles = (n_rows + R - 1) / R;
    for (int64_t tile = cta_in_slab; tile < n_tiles; tile += n_ctas) {
      const int64_t r0 = tile * R;
      const int rows_in_tile = int(min(int64_t(R), n_rows - r0));

      // ---------------- A. predicates and survivor compaction
      const int n_surv = tile_survivors(tb, r0, rows_in_tile, R, vec, surv, sint);
      my_survivors += n_surv;

      // ---------------- B. per key column: aggregate equal keys, hash, update
      for (int kc = 0; kc < n_keycols; kc++) {
        const int c = cols_list[kc];
        if (A.agg && tb->agg[c] >= 0) {  // hashed by the column's aggregated items when active
          int64_t kmin, range;
          if (agg_active(A.agg[tb->agg[c]], tb->agg[c], A.ws, &kmin, &range)) continue;
        }
        const void* kbase = tb->col[c];
        const int32_t kdt = tb->dtype[c];
        int n_entries = n_surv;
        if (DEDUPE) {
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
                atomicAdd(&mcnt[slot], __popc(peers));
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
        hash_entries(kc, n_entries, kbase, kdt, r0, DEDUPE);
        __syncthreads();  // map / survivor list reused next
      }
    }
  }

  // ---------------- C. flush private counters, count survivors once per table
  if (!GLOBAL) {
    for (int j = tid; j < npairs * w; j += T) {
      const int32_t v = cnt[j];
      if (v) atomicAdd(gcnt + j, v);
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
// Smallest and largest key of every aggregated column over all its rows (a bound on the
// survivors' keys).  Column a is read by CTAs [stat_cta0, stat_cta0 + stat_ncta), each
// one contiguous slice, four 4-row loads in flight per thread.
constexpr int kStatThreads = 256;

__global__ void __launch_bounds__(kStatThreads) k_agg_stats(const __grid_constant__ BuildArgs A) {
  __shared__ long long red[2][kStatThreads / 32];
  int ai = 0;
  while (ai + 1 < A.n_agg && A.agg[ai + 1].stat_cta0 <= int(blockIdx.x)) ai++;
  const AggCol ac = A.agg[ai];
  const DevTable* tb = A.tables + ac.table;
  const void* base = tb->col[ac.col];
  const int32_t dt = tb->dtype[ac.col];
  const bool vec = tb->vec_ok != 0;
  const int64_t n = tb->n_rows;
  const int64_t per = ((n + ac.stat_ncta - 1) / ac.stat_ncta + 15) & ~int64_t(15);  // rows per CTA, x16
  const int64_t r_begin = min(n, per * (int64_t(blockIdx.x) - ac.stat_cta0)), r_end = min(n, r_begin + per);
  int64_t mn = INT64_MAX, mx = INT64_MIN;
  for (int64_t r = r_begin + 16 * int64_t(threadIdx.x); r < r_end; r += 16 * int64_t(blockDim.x)) {
    int64_t v[4][4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int nvalid = int(max(int64_t(0), min(int64_t(4), r_end - (r + 4 * u))));
      load4(base, dt, r + 4 * u, nvalid, vec, v[u]);
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (k >= nvalid) v[u][k] = v[0][0];  // padding repeats row r, valid inside the loop
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int k = 0; k < 4; k++) {
        mn = min(mn, v[u][k]);
        mx = max(mx, v[u][k]);
      }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mn = min(mn, (int64_t)__shfl_down_sync(0xffffffffu, (long long)mn, off));
    mx = max(mx, (int64_t)__shfl_down_sync(0xffffffffu, (long long)mx, off));
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][warp] = mn;
    red[1][warp] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < int(blockDim.x >> 5); q++) {
      mn = min(mn, int64_t(red[0][q]));
      mx = max(mx, int64_t(red[1][q]));
    }
    if (mx >= mn) {
      unsigned long long* st = reinterpret_cast<unsigned long long*>(A.ws) + 2 * int64_t(ai);
      atomicMax(st, (unsigned long long)enc_max(mx));
      atomicMax(st + 1, (unsigned long long)enc_min(mn));
    }
  }
}

// Clears the used part [0, range) of every active column's count array; grid.y = column.
__global__ void __launch_bounds__(256) k_agg_zero(const __grid_constant__ BuildArgs A) {
  const int ai = int(blockIdx.y);
  const AggCol ac = A.agg[ai];
  int64_t kmin, range;
  if (!agg_active(ac, ai, A.ws, &kmin, &range)) return;
  int4* c4 = reinterpret_cast<int4*>(A.ws + ac.off);  // 256-byte aligned
  const int64_t n4 = (range + 3) / 4;                 // within cap rounded up to 64 entries
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x)
    c4[i] = make_int4(0, 0, 0, 0);
}

// Per tile of a table with aggregated columns: survivors (phase A), then for every active
// column the tile's keys reduced in a shared-memory map and one global atomic per
// occupied slot.  A slot packs (key - min) in its high 32 bits and the tile count in its
// low 32 bits (a count never exceeds the tile's rows), so an insert is one atomic: a CAS
// that claims an empty slot with the count, or an add to a slot holding the key.  Equal
// keys of a warp are inserted once, by their lowest lane (__match_any_sync).  The flush
// also empties the slots, so the map is cleared once per CTA.
__global__ void __launch_bounds__(1024) k_agg_count(const __grid_constant__ BuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const CountItem it = A.cnt_items[A.cnt_cta_item[blockIdx.x]];
  const DevTable* tb = A.tables + it.table;
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
  const int R = A.tile_rows, M = A.map_slots;
  unsigned char* sp = smem;
  unsigned long long* slot64 = reinterpret_cast<unsigned long long*>(sp);
  sp += align16(sizeof(unsigned long long) * size_t(M));
  uint16_t* surv = reinterpret_cast<uint16_t*>(sp);
  sp += align16(sizeof(uint16_t) * R);
  int32_t* sint = reinterpret_cast<int32_t*>(sp);
  constexpr unsigned long long kEmpty = ~0ull;  // key part 0xFFFFFFFF is never an index: cap <= 2^31 - 1
  const int64_t n_rows = tb->n_rows;
  const int64_t n_tiles = (n_rows + R - 1) / R;
  const int filtered = tb->filtered;
  const bool vec = tb->vec_ok != 0;
  const int cta = int(blockIdx.x) - it.first_cta;
  const uint32_t mmask = uint32_t(M - 1);
  for (int s = tid; s < M; s += T) slot64[s] = kEmpty;
  __syncthreads();
  for (int64_t tile = cta; tile < n_tiles; tile += it.n_ctas) {
    const int64_t r0 = tile * R;
    const int rows_in_tile = int(min(int64_t(R), n_rows - r0));
    const int n_surv = tile_survivors(tb, r0, rows_in_tile, R, vec, surv, sint);
    for (int c = 0; c < tb->n_cols; c++) {
      const int ai = tb->agg[c];
      if (ai < 0) continue;
      int64_t kmin, range;
      if (!agg_active(A.agg[ai], ai, A.ws, &kmin, &range)) continue;  // block-uniform
      int32_t* cnts = reinterpret_cast<int32_t*>(A.ws + A.agg[ai].off);
      const void* kbase = tb->col[c];
      const int32_t kdt = tb->dtype[c];
      for (int base = 0; base < n_surv; base += T) {  // block-uniform trip count
        const int e = base + tid;
        const bool valid = e < n_surv;
        uint32_t x = 0xFFFFFFFFu;
        if (valid) x = uint32_t(load1(kbase, kdt, r0 + (filtered ? surv[e] : e)) - kmin);  // < range <= cap
        const unsigned peers = __match_any_sync(0xffffffffu, x);
        if (!valid || lane != __ffs(peers) - 1) continue;
        const unsigned long long cnt = (unsigned long long)__popc(peers);
        uint32_t slot = map_slot(x, mmask);
        bool done = false;
        for (int probe = 0; probe < M && !done; probe++) {
          const unsigned long long cur = slot64[slot];
          if (uint32_t(cur >> 32) == x) {
            atomicAdd(&slot64[slot], cnt);
            done = true;
          } else if (cur == kEmpty) {
            const unsigned long long prev = atomicCAS(&slot64[slot], kEmpty, ((unsigned long long)x << 32) | cnt);
            if (prev == kEmpty) {
              done = true;
            } else if (uint32_t(prev >> 32) == x) {
              atomicAdd(&slot64[slot], cnt);
              done = true;
            }
          }
          if (!done) slot = (slot + 1) & mmask;
        }
        if (!done) set_status(A.status, CMP_ETIMEOUT);  // unreachable: M > tile rows
      }
      __syncthreads();
      for (int s = tid; s < M; s += T) {
        const unsigned long long v = slot64[s];
        if (v != kEmpty) {
          atomicAdd(cnts + uint32_t(v >> 32), int32_t(uint32_t(v)));
          slot64[s] = kEmpty;
        }
      }
      __syncthreads();  // map reused next
    }
  }
}

size_t agg_count_smem_bytes(const BuildShape& s) {
  return align16(sizeof(unsigned long long) * size_t(s.map_slots)) + align16(sizeof(uint16_t) * s.tile_rows) +
         sizeof(int32_t) * 40;
}

cudaError_t launch_agg(const BuildArgs& a, const BuildShape& s, int32_t stat_grid, int32_t cnt_grid,
                       cudaStream_t st) {
  if (a.n_agg <= 0) return cudaSuccess;
  k_agg_stats<<<unsigned(stat_grid), kStatThreads, 0, st>>>(a);
  const dim3 g(unsigned(std::max(1, 4 * sm_count() / std::max(1, a.n_agg))), unsigned(a.n_agg));
  k_agg_zero<<<g, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || cnt_grid <= 0) return e;
  const size_t smem = agg_count_smem_bytes(s);
  e = cudaFuncSetAttribute(k_agg_count, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  k_agg_count<<<unsigned(cnt_grid), s.threads, smem, st>>>(a);
  return cudaGetLastError();
}

__global__ void k_zero_spans(const ZeroSpan* __restrict__ spans, int32_t n) {
  // one block-stride pass per span; spans are 4-byte multiples
  for (int32_t s = blockIdx.y; s < n; s += gridDim.y) {
    const ZeroSpan z = spans[s];
    uint32_t* p = reinterpret_cast<uint32_t*>(z.ptr);
    const int64_t words = z.bytes / 4;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < words; i += int64_t(gridDim.x) * blockDim.x)
      p[i] = 0;
  }
}

cudaError_t launch_zero_spans(const ZeroSpan* spans_dev, int32_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(64, unsigned(n < 1024 ? n : 1024));
  k_zero_spans<<<grid, 256, 0, st>>>(spans_dev, n);
  return cudaGetLastError();
}

}  // namespace cmpk
