// Shared-memory counter slabs of the batched build's hashing kernels (unique-key rows and
// presence-bitmap domains): int32 counters, or two 16-bit halves per 32-bit word.  Each
// half starts at 2^15.  An atomic add on the word returns its old value, so the thread
// whose add carries a half past 0xFFFF or borrows it below 0 sees it and no other: it adds
// +-2^16 for that half straight to the global counter and, for a carry out of the low half
// into the high one, takes it back with a second add on the word (whose own wrap it checks
// the same way).  At the end each half minus 2^15 is added to the global counter; the
// counters are therefore exact whatever the number of updates or their order.
#pragma once

#include "internal.cuh"

namespace cmpk {
namespace {

constexpr uint32_t kHalfBias = 0x8000u;
constexpr uint32_t kWordBias = 0x80008000u;

// Slow path of a packed update: `old` is the word before this thread's add of (dl, dh) to
// its (low, high) halves; g2 = global counters of the word's even and odd bucket.
__device__ __noinline__ void pack16_wrap(uint32_t* word, int32_t* g2, int dl, int dh, uint32_t old, bool has_hi) {
  for (int guard = 0; guard < 2; guard++) {  // a take-back (dl = 0) never carries again
    const int lo = int(old & 0xFFFFu) + dl;
    const int cl = lo > 0xFFFF ? 1 : (lo < 0 ? -1 : 0);
    const int hi = int(old >> 16) + dh + cl;
    const int ch = hi > 0xFFFF ? 1 : (hi < 0 ? -1 : 0);
    if (cl) red_add(g2, cl * 65536);
    if (ch && has_hi) red_add(g2 + 1, ch * 65536);
    if (!cl) return;
    dl = 0;  // the carry (cl) reached the high half: take it back
    dh = -cl;
    old = atomicAdd(word, uint32_t(dh) << 16);
  }
}

template <bool PACK16>
__device__ __forceinline__ void counter_add(uint32_t* cs, int32_t* g, uint32_t h, int sg, uint32_t w) {
  if (PACK16) {
    const uint32_t odd = h & 1u;
    uint32_t* wd = cs + (h >> 1);
    const uint32_t sh = odd << 4;
    const uint32_t old = atomicAdd(wd, uint32_t(sg) << sh);
    // only the updated half can wrap (the other one changes only through its carry)
    if ((((old >> sh) & 0xFFFFu) - 1u) >= 0xFFFEu)
      pack16_wrap(wd, g + (h & ~1u), odd ? 0 : sg, odd ? sg : 0, old, (h | 1u) < w);
  } else {
    red_add_shared(reinterpret_cast<int32_t*>(cs) + h, sg);
  }
}

}  // namespace
}  // namespace cmpk
