// Device helpers shared by the estimate kernels: checked int128 arithmetic, block-wide
// sums and scans, and ranks in presorted magnitude rows.
#pragma once

#include "estimate.cuh"

namespace cmpk {
namespace {

// ---------------------------------------------------------------- checked int128
__device__ __forceinline__ bool add_ovf(i128 a, i128 b, i128* r) {
  const i128 s = i128(u128(a) + u128(b));
  *r = s;
  return ((a ^ s) & (b ^ s)) < 0;
}

__device__ __forceinline__ bool fits64(i128 v) { return v == i128(int64_t(v)); }

// a * b for |b| <= 2^63 (b from a stored int64 or int32 value), overflow-checked.
__device__ __forceinline__ bool mul_ovf_64(i128 a, int64_t b, i128* r) {
  if (fits64(a)) {
    const int64_t x = int64_t(a);
    const uint64_t lo = uint64_t(x) * uint64_t(b);
    const int64_t hi = __mul64hi(x, b);
    *r = i128((u128(uint64_t(hi)) << 64) | lo);
    return false;
  }
  // |a| * |b| = (ah * |b|) 2^64 + al * |b| with ah = |a| >> 64 < 2^63
  const bool neg = (a < 0) != (b < 0);
  const u128 ua = a < 0 ? u128(0) - u128(a) : u128(a);
  const uint64_t ub = b < 0 ? uint64_t(0) - uint64_t(b) : uint64_t(b);
  const uint64_t ah = uint64_t(ua >> 64), al = uint64_t(ua);
  const u128 hi = u128(ah) * ub;          // must stay below 2^63 after the carry
  const u128 lo = u128(al) * ub;
  const u128 top = hi + (lo >> 64);
  const bool ovf = (top >> 63) != 0 && !(neg && top == (u128(1) << 63) && uint64_t(lo) == 0);
  const u128 mag = (top << 64) | uint64_t(lo);
  *r = neg ? i128(u128(0) - mag) : i128(mag);
  return ovf;
}

__device__ __forceinline__ bool mul_ovf(i128 a, i128 b, i128* r);
__device__ __forceinline__ bool mul_s(i128 a, int64_t b, i128* r) { return mul_ovf_64(a, b, r); }
__device__ __forceinline__ bool mul_s(i128 a, i128 b, i128* r) { return mul_ovf(a, b, r); }

__device__ __forceinline__ bool mul_ovf(i128 a, i128 b, i128* r) {
  if (fits64(a) && fits64(b)) {  // |a|, |b| <= 2^63: the product fits int128 exactly
    const int64_t x = int64_t(a), y = int64_t(b);
    const uint64_t lo = uint64_t(x) * uint64_t(y);
    const int64_t hi = __mul64hi(x, y);
    *r = i128((u128(uint64_t(hi)) << 64) | lo);
    return false;
  }
  const bool neg = (a < 0) != (b < 0);
  const u128 ua = a < 0 ? u128(0) - u128(a) : u128(a);
  const u128 ub = b < 0 ? u128(0) - u128(b) : u128(b);
  const uint64_t a1 = uint64_t(ua >> 64), a0 = uint64_t(ua), b1 = uint64_t(ub >> 64), b0 = uint64_t(ub);
  bool ovf = false;
  u128 mag;
  if (a1 == 0 && b1 == 0) {
    mag = u128(a0) * b0;
  } else if (a1 && b1) {
    ovf = true;
    mag = 0;
  } else {
    const u128 cross = a1 ? u128(a1) * b0 : u128(b1) * a0;
    const u128 low = u128(a0) * b0;
    if (uint64_t(cross >> 64)) ovf = true;
    const u128 hi_part = cross << 64;
    mag = low + hi_part;
    if (mag < low) ovf = true;
  }
  const u128 lim = u128(1) << 127;
  if (neg ? mag > lim : mag >= lim) ovf = true;
  *r = neg ? i128(u128(0) - mag) : i128(mag);
  return ovf;
}

// exact (a + b) / 2 rounded once (the sum may need 129 bits)
__device__ __forceinline__ double mean2_to_double(i128 a, i128 b) {
  i128 s;
  if (!add_ovf(a, b, &s)) return i128_to_double(s) * 0.5;
  // same signs overflowed: |a| + |b| = 2^128 * top + low
  const bool neg = a < 0;
  const u128 ua = neg ? u128(0) - u128(a) : u128(a);
  const u128 ub = neg ? u128(0) - u128(b) : u128(b);
  const u128 low = ua + ub;
  const uint32_t top = low < ua ? 1u : 0u;
  return mag_to_double(neg, top, low) * 0.5;
}

// first position q in sorted a[0..w) with a[q] > tau (strict) or a[q] >= tau
__device__ __forceinline__ int rank_of(const uint32_t* __restrict__ a, int w, uint32_t tau, bool strict) {
  int lo = 0, hi = w;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const uint32_t v = __ldg(a + mid);
    if (strict ? v <= tau : v < tau) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

struct BlockScratch {
  i128* sh_i128;    // [33]
  int32_t* sh_flag;  // [1]
};

// block-wide sum of one int128 per thread (checked); result broadcast
__device__ i128 block_sum(i128 v, bool* ovf, BlockScratch& bs) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  bool o = false;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int64_t lo = __shfl_down_sync(0xffffffffu, int64_t(v), off);
    const int64_t hi = __shfl_down_sync(0xffffffffu, int64_t(v >> 64), off);
    const i128 other = (i128(hi) << 64) | i128(uint64_t(lo));
    i128 r;
    const bool ob = add_ovf(v, other, &r);
    if (lane + off < 32) {
      o |= ob;
      v = r;
    }
  }
  if (lane == 0) bs.sh_i128[warp] = v;
  if (o) atomicOr(bs.sh_flag, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    i128 t = 0;
    bool oo = false;
    for (int i = 0; i < nw; i++) oo |= add_ovf(t, bs.sh_i128[i], &t);
    bs.sh_i128[32] = t;
    if (oo) atomicOr(bs.sh_flag, 1);
  }
  __syncthreads();
  const i128 r = bs.sh_i128[32];
  *ovf |= bs.sh_flag[0] != 0;
  __syncthreads();
  return r;
}

// Whether an exact value fits the storage type of the scratch arrays.
__device__ __forceinline__ bool store_fits(i128 v, int64_t*) { return v == i128(int64_t(v)); }
__device__ __forceinline__ bool store_fits(i128, i128*) { return true; }

// In-place inclusive scan of a[0..n) (forward) or suffix scan (reverse).  Sums are exact
// in int128 (bit 0 of the flag on overflow); a stored value that does not fit S sets
// bit 1 (the item is then recomputed with int128 storage).
// int64 storage: partial sums stay in int64 (overflow only flags bit 1: the item is then
// recomputed with int128 storage, so no int128 work is needed here).
__device__ __forceinline__ bool add64_ovf(int64_t a, int64_t b, int64_t* r) {
  const int64_t s = int64_t(uint64_t(a) + uint64_t(b));
  *r = s;
  return ((a ^ s) & (b ^ s)) < 0;
}

__device__ void block_scan(int64_t* a, int n, bool reverse, BlockScratch& bs) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int per = (n + T - 1) / T;
  const int b = tid * per, e = min(n, b + per);
  int64_t s = 0;
  bool o = false;
  if (reverse) {
    for (int q = b; q < e; q++) o |= add64_ovf(s, a[n - 1 - q], &s);
  } else {
    for (int q = b; q < e; q++) o |= add64_ovf(s, a[q], &s);
  }
  const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  int64_t incl = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t other = __shfl_up_sync(0xffffffffu, incl, off);
    int64_t r;
    const bool ob = add64_ovf(incl, other, &r);
    if (lane >= off) {
      o |= ob;
      incl = r;
    }
  }
  int64_t* sh = reinterpret_cast<int64_t*>(bs.sh_i128);
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (tid == 0) {
    int64_t t = 0;
    bool oo = false;
    for (int i = 0; i < nw; i++) {
      const int64_t v = sh[i];
      sh[i] = t;
      oo |= add64_ovf(t, v, &t);
    }
    if (oo) atomicOr(bs.sh_flag, 2);
  }
  __syncthreads();
  int64_t run;
  o |= add64_ovf(sh[warp], incl - s, &run);
  if (reverse) {
    for (int q = b; q < e; q++) {
      o |= add64_ovf(run, a[n - 1 - q], &run);
      a[n - 1 - q] = run;
    }
  } else {
    for (int q = b; q < e; q++) {
      o |= add64_ovf(run, a[q], &run);
      a[q] = run;
    }
  }
  if (o) atomicOr(bs.sh_flag, 2);
  __syncthreads();
}

template <typename S>
__device__ void block_scan(S* a, int n, bool reverse, BlockScratch& bs) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int per = (n + T - 1) / T;
  const int b = tid * per, e = min(n, b + per);
  i128 s = 0;
  bool o = false;
  for (int q = b; q < e; q++) o |= add_ovf(s, i128(a[reverse ? n - 1 - q : q]), &s);
  // exclusive scan of thread sums (thread order = scan order)
  const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  i128 incl = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t lo = __shfl_up_sync(0xffffffffu, int64_t(incl), off);
    const int64_t hi = __shfl_up_sync(0xffffffffu, int64_t(incl >> 64), off);
    const i128 other = (i128(hi) << 64) | i128(uint64_t(lo));
    i128 r;
    const bool ob = add_ovf(incl, other, &r);
    if (lane >= off) {
      o |= ob;
      incl = r;
    }
  }
  if (lane == 31) bs.sh_i128[warp] = incl;
  __syncthreads();
  if (tid == 0) {
    i128 t = 0;
    bool oo = false;
    for (int i = 0; i < nw; i++) {
      const i128 v = bs.sh_i128[i];
      bs.sh_i128[i] = t;
      oo |= add_ovf(t, v, &t);
    }
    if (oo) atomicOr(bs.sh_flag, 1);
  }
  __syncthreads();
  i128 run;
  o |= add_ovf(bs.sh_i128[warp], incl - s, &run);  // incl - s cannot overflow: it is a partial sum
  bool so = false;
  for (int q = b; q < e; q++) {
    const int idx = reverse ? n - 1 - q : q;
    o |= add_ovf(run, i128(a[idx]), &run);
    so |= !store_fits(run, a);
    a[idx] = S(run);
  }
  if (o) atomicOr(bs.sh_flag, 1);
  if (so) atomicOr(bs.sh_flag, 2);
  __syncthreads();
}

}  // namespace
}  // namespace cmpk
