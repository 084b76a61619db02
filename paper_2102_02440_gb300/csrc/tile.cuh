// Device helpers of the table scans (1-D and partitioned builds): column loads and the
// pushed-down predicate pass over one tile of rows (Sec. 2 "Partitioned query execution").
#pragma once

#include "internal.cuh"

namespace cmpk {
namespace {

__device__ __forceinline__ int64_t load1(const void* base, int32_t dtype, int64_t row) {
  return dtype == CMP_I32 ? int64_t(__ldg(reinterpret_cast<const int32_t*>(base) + row))
                          : int64_t(__ldg(reinterpret_cast<const long long*>(base) + row));
}

// Bulk prefetch of [p, p + bytes) into L2 (cp.async.bulk.prefetch: no registers, no shared
// memory, no completion to wait for), shrunk to its 16-byte-aligned interior so that no
// byte outside the range is touched; pieces of at most 32 KB.
__device__ __forceinline__ void l2_prefetch(const void* p, int64_t bytes) {
  if (bytes <= 0) return;
  const size_t g = __cvta_generic_to_global(p);
  size_t a = (g + 15) & ~size_t(15);
  const size_t e = (g + size_t(bytes)) & ~size_t(15);
  for (; a < e; a += 32768) {
    const uint32_t n = uint32_t(e - a < 32768 ? e - a : 32768);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
  }
}

// One bulk L2 prefetch of [p, p + bytes): p 16-byte aligned, bytes a multiple of 16 and at
// most 2^20 (the caller guarantees both).
__device__ __forceinline__ void l2_prefetch_exact(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(bytes) : "memory");
}

// L2 prefetch of rows [r0, r1) (clamped to the table) of the columns a scan of table tb
// reads: its predicate columns, then (when with_keys) the key columns selected by
// key_cols (bit c: column c).  Thread `who` of `nwho` takes every nwho-th column.
__device__ __forceinline__ void prefetch_rows(const DevTable* tb, uint32_t key_cols, int64_t r0, int64_t r1,
                                              int who, int nwho) {
  r1 = r1 < tb->n_rows ? r1 : tb->n_rows;
  if (r0 >= r1) return;
  const int np = tb->n_preds, nc = tb->n_cols;
  for (int j = who; j < np + nc; j += nwho) {
    const int c = j < np ? tb->pred[j].col : j - np;
    if (j >= np && !((key_cols >> c) & 1u)) continue;
    const int es = tb->dtype[c] == CMP_I32 ? 4 : 8;
    l2_prefetch(static_cast<const char*>(tb->col[c]) + r0 * es, (r1 - r0) * es);
  }
}

// 4 consecutive rows starting at `row` (row % 4 == 0); nvalid in 0..4.
__device__ __forceinline__ void load4(const void* base, int32_t dtype, int64_t row, int nvalid, bool vec,
                                      int64_t v[4]) {
  if (dtype == CMP_I32) {
    const int32_t* p = reinterpret_cast<const int32_t*>(base) + row;
    if (vec && nvalid == 4) {
      const int4 q = __ldg(reinterpret_cast<const int4*>(p));
      v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; k++) v[k] = k < nvalid ? int64_t(__ldg(p + k)) : 0;
    }
  } else {
    const long long* p = reinterpret_cast<const long long*>(base) + row;
    if (vec && nvalid == 4) {
      const longlong2 a = __ldg(reinterpret_cast<const longlong2*>(p));
      const longlong2 b = __ldg(reinterpret_cast<const longlong2*>(p + 2));
      v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    } else {
#pragma unroll
      for (int k = 0; k < 4; k++) v[k] = k < nvalid ? int64_t(__ldg(p + k)) : 0;
    }
  }
}

__device__ __forceinline__ bool pred_holds(const DevPred& q, int64_t v) {
  if (q.op == CMP_RANGE) return q.lo <= v && v < q.hi;
  if (q.op == CMP_EQ) return v == q.lo;
  if (v < 0 || v >= q.nbits) return false;
  return (__ldg(q.bitmap + (v >> 5)) >> (v & 31)) & 1u;
}

// A RANGE or EQ predicate on an int32 column as one 32-bit unsigned comparison: v holds iff
// uint32(v - lo) < span, with [lo, lo + span) the predicate's interval clipped to int32;
// all = every int32 value holds (an interval of 2^32 values), none when it is empty.
struct PredI32 {
  uint32_t lo, span;
  int32_t all;
};
__device__ __forceinline__ PredI32 pred_i32(const DevPred& q) {
  int64_t L = q.lo, H = q.op == CMP_EQ ? q.lo + 1 : q.hi;  // [L, H)
  if (q.op == CMP_EQ && q.lo == INT64_MAX) H = INT64_MAX;  // no int32 value equals it anyway
  L = L < INT32_MIN ? INT32_MIN : L;
  H = H > int64_t(INT32_MAX) + 1 ? int64_t(INT32_MAX) + 1 : H;
  PredI32 r;
  r.all = L == INT32_MIN && H == int64_t(INT32_MAX) + 1;
  r.lo = uint32_t(L);
  r.span = H > L && !r.all ? uint32_t(H - L) : 0u;  // < 2^32 unless all
  return r;
}
__device__ __forceinline__ bool i32_holds(const PredI32& q, int32_t v) {
  return q.all || uint32_t(v) - q.lo < q.span;
}

// A predicate in registers: RANGE [lo, hi) and EQ (= [lo, lo + 1)) as one unsigned
// comparison, v - lo < span in 64-bit arithmetic (span = 0: nothing holds); IN as its
// bitmap.  The same truth value as pred_holds for every int64 v.
struct PredReg {
  uint64_t lo, span;
  const uint32_t* bitmap;  // IN only
  int64_t nbits;
  int32_t in;
};
__device__ __forceinline__ PredReg pred_reg(const DevPred& q) {
  PredReg r;
  r.in = q.op != CMP_RANGE && q.op != CMP_EQ;
  r.lo = uint64_t(q.lo);
  r.span = q.op == CMP_EQ ? 1 : (q.op == CMP_RANGE && q.hi > q.lo ? uint64_t(q.hi) - uint64_t(q.lo) : 0);
  r.bitmap = q.bitmap;
  r.nbits = q.nbits;
  return r;
}
__device__ __forceinline__ bool reg_holds(const PredReg& q, int64_t v) {
  if (!q.in) return uint64_t(v) - q.lo < q.span;
  if (v < 0 || v >= q.nbits) return false;
  return (__ldg(q.bitmap + (v >> 5)) >> (v & 31)) & 1u;
}

// Phase A of one tile: the row sample and the predicate conjunction over rows [r0, r0 +
// rows_in_tile), the survivors' offsets compacted into surv[] (warp scan, one shared atomic
// per warp).  An unfiltered table returns rows_in_tile without writing surv[].
// Returns the survivor count.  Block-wide: every thread calls it; sint[0] is the tail.
__device__ int tile_survivors(const DevTable* tb, int64_t r0, int rows_in_tile, int R, bool vec, uint16_t* surv,
                              int32_t* sint) {
  const int n_preds = tb->n_preds;
  if (!tb->filtered) return rows_in_tile;
  const uint64_t keep = tb->sample_keep, seed = tb->sample_seed;
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
  if (tid == 0) sint[0] = 0;
  __syncthreads();
  const int iters = (R + 4 * T - 1) / (4 * T);
  for (int it = 0; it < iters; it++) {
    const int base = 4 * (tid + it * T);
    const int nvalid = max(0, min(4, rows_in_tile - base));
    uint32_t m = (1u << nvalid) - 1u;
    if (keep) {  // row sample: one SplitMix64 trial per row of the table
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (((m >> k) & 1u) && splitmix64_at(seed, uint64_t(r0 + base + k)) >= keep) m &= ~(1u << k);
    }
    for (int q = 0; q < n_preds && m; q++) {
      const DevPred& pq = tb->pred[q];
      int64_t v[4];
      load4(tb->col[pq.col], tb->dtype[pq.col], r0 + base, nvalid, vec, v);
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (!pred_holds(pq, v[k])) m &= ~(1u << k);
    }
    const int c = __popc(m);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int wbase = 0;
    if (lane == 31) wbase = atomicAdd(&sint[0], incl);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    int pos = wbase + incl - c;
#pragma unroll
    for (int k = 0; k < 4; k++)
      if ((m >> k) & 1u) surv[pos++] = uint16_t(base + k);
  }
  __syncthreads();
  return sint[0];
}


}  // namespace
}  // namespace cmpk
