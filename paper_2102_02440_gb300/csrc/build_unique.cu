// Unique key columns of the batched build (Sec. 3.2 "Fast-AGMS Sketches": every selected
// tuple adds xi_i(key) to bucket h_i(key) of row i).  A column declared unique (a primary
// key) has no repeated keys, so counting survivors per key first (key aggregation) saves
// no hashing.  Its tuples are hashed once per (sketch, row) pair with the pair's counters
// held in shared memory, so the updates are shared-memory atomics instead of L2 atomics.
//
// A slab is a set of the column's pairs whose counters fit the shared-memory budget:
//  - int32 counters, several pairs per slab (w small enough); the key's powers are
//    computed once per key and shared by the slab's pairs;
//  - one pair per slab as two 16-bit halves per 32-bit word (w up to 2x the int32 limit,
//    e.g. 65536 buckets in 128 KB), with every carry and borrow of a half added to the
//    global counter (slab.cuh), so that the counters stay exact.
// An item is one slab over a range of the table's rows (whole tiles); the plan gives each
// CTA a list of items of about equal row counts, CTAs of the same column's slabs covering
// the same row ranges (their key reads meet in L2).  The kernel has no inter-CTA waits.
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.cuh"
#include "slab.cuh"
#include "tile.cuh"

namespace cmpk {

constexpr int kUniqThreads = 512;
// keys per thread and step (even): two keep the kernel within 64 registers, so that one
// CTA of it and one of the counting pass fit on an SM together
constexpr int KPT = 2;


size_t uniq_smem_bytes(int32_t words, int32_t tile_rows) {
  return align16(sizeof(uint32_t) * size_t(words)) + align16(sizeof(uint16_t) * size_t(tile_rows)) +
         sizeof(int32_t) * 40;
}

template <bool PACK16, bool POW2>
__global__ void __launch_bounds__(kUniqThreads, 2) k_uniq_hash(const __grid_constant__ BuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PairParam prm[kUniqMaxPairs];
  __shared__ int32_t* grow[kUniqMaxPairs];
  const int tid = threadIdx.x, T = blockDim.x;
  const uint32_t w = uint32_t(A.w);
  const int R = A.tile_rows;
  uint32_t* cs = reinterpret_cast<uint32_t*>(smem);
  uint16_t* surv = reinterpret_cast<uint16_t*>(smem + align16(sizeof(uint32_t) * size_t(A.u_words)));
  int32_t* sint = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(surv) +
                                            align16(sizeof(uint16_t) * size_t(R)));
  // items of this CTA: [cta_item[blockIdx.x], cta_item[blockIdx.x + 1]) of the unique items
  const int64_t i_begin = A.u_cta_item[blockIdx.x], i_end = A.u_cta_item[blockIdx.x + 1];
  const int words = A.u_words;
  for (int j = tid; j < words; j += T) cs[j] = PACK16 ? kWordBias : 0u;
  int cur = -1;     // slab whose counters are in shared memory (block-uniform)
  int n_pairs = 0;
  auto flush = [&]() {
    __syncthreads();
    if (PACK16) {
      int32_t* g = grow[0];
      for (int j = tid; j < words; j += T) {
        const uint32_t v = cs[j];
        const int32_t lo = int32_t(v & 0xFFFFu) - int32_t(kHalfBias), hi = int32_t(v >> 16) - int32_t(kHalfBias);
        if (lo) red_add(g + 2 * j, lo);
        if (hi && uint32_t(2 * j + 1) < w) red_add(g + 2 * j + 1, hi);
        cs[j] = kWordBias;
      }
    } else {
      for (int j = tid; j < n_pairs * int(w); j += T) {
        const int32_t v = int32_t(cs[j]);
        if (v) red_add(grow[j / int(w)] + (j % int(w)), v);
        cs[j] = 0;
      }
    }
    __syncthreads();
  };
  for (int64_t ii = i_begin; ii < i_end; ii++) {
    const UniqItem it = A.uitem[ii];
    const UniqSlab& sl = A.uslab[it.slab];
    const DevTable* tb = A.tables + sl.table;
    if (it.slab != cur) {
      if (cur >= 0) flush();
      if (tid < sl.n_pairs) {
        const int pair = sl.pair[tid];
        const int s = pair / A.d, i = pair % A.d;
        prm[tid] = make_pair_param(A.hash[size_t(tb->edge_id[s]) * A.d + i]);
        grow[tid] = tb->counters + size_t(pair) * w;
      }
      cur = it.slab;
      n_pairs = sl.n_pairs;
      __syncthreads();
    }
    const void* kbase = tb->col[sl.col];
    const int32_t kdt = tb->dtype[sl.col];
    const bool vec = tb->vec_ok != 0;
    const int filtered = tb->filtered;
    int64_t my_surv = 0;
    // KPT keys per thread and step: independent hash chains sharing the parameters; their
    // counter updates are issued before any of their results is examined
    // (packed slabs hold one pair: the Horner form, no shared powers; int32 slabs share the
    // key's powers x^2, x^3 among their pairs)
    auto hashk = [&](const int64_t (&k)[KPT], int nv) {
      KeyPow kp[KPT];
      KeyX kx[KPT];
      uint32_t hi_or = 0;
      // keys in [0, p) are their own residue (every non-negative key below 2^61)
      bool in_field = true;
#pragma unroll
      for (int q = 0; q < KPT; q++) in_field &= uint64_t(k[q]) < kP61;
      in_field = __all_sync(__activemask(), in_field);
#pragma unroll
      for (int q = 0; q < KPT; q++) {
        const uint64_t x = in_field ? uint64_t(k[q]) : key_field(k[q]);
        if (PACK16) kx[q] = key_x(x);
        else kp[q] = key_powers(x);
        hi_or |= PACK16 ? kx[q].hi : kp[q].x.hi;
      }
      auto run = [&](auto smallx) {
        constexpr bool SX = decltype(smallx)::value;
        for (int p = 0; p < n_pairs; p++) {
          const PairParam prm_p = prm[p];
          const uint64_t c2 = prm_p.c2_lo | (uint64_t(prm_p.c2_hi) << 31);
          const uint64_t c1 = prm_p.c1_lo | (uint64_t(prm_p.c1_hi) << 31);
          uint32_t h[KPT];
          int sg[KPT];
#pragma unroll
          for (int q = 0; q < KPT; q++) {
            if (PACK16) {
              h[q] = cw_bucket_h<POW2, SX>(prm_p, kx[q], w, A.m31, A.m4);
              sg[q] = cw_sign_h<SX>(prm_p, kx[q], c2, c1, A.m31, A.m4);
            } else {
              h[q] = cw_bucket<POW2, SX>(prm_p, kp[q], w);
              sg[q] = cw_sign<SX>(prm_p, kp[q]);
            }
          }
          if (PACK16) {
            uint32_t old[KPT];
#pragma unroll
            for (int q = 0; q < KPT; q++)
              if (q < nv) old[q] = atomicAdd(cs + (h[q] >> 1), uint32_t(sg[q]) << ((h[q] & 1u) << 4));
#pragma unroll
            for (int q = 0; q < KPT; q++)
              if (q < nv && (((old[q] & 0xFFFFu) - 1u) >= 0xFFFEu || ((old[q] >> 16) - 1u) >= 0xFFFEu)) {
                const uint32_t odd = h[q] & 1u;
                pack16_wrap(cs + (h[q] >> 1), grow[0] + (h[q] & ~1u), odd ? 0 : sg[q], odd ? sg[q] : 0, old[q],
                            (h[q] | 1u) < w);
              }
          } else {
            int32_t* c = reinterpret_cast<int32_t*>(cs) + size_t(p) * w;
#pragma unroll
            for (int q = 0; q < KPT; q++)
              if (q < nv) red_add_shared(c + h[q], sg[q]);
          }
        }
      };
      if (__all_sync(__activemask(), hi_or == 0)) run(std::true_type{});
      else run(std::false_type{});
    };
    for (int64_t r0 = it.row_begin; r0 < it.row_end; r0 += R) {
      const int rows_in_tile = int(min(int64_t(R), it.row_end - r0));
      if (filtered) {
        const int n_surv = tile_survivors(tb, r0, rows_in_tile, R, vec, surv, sint);
        my_surv += n_surv;
        for (int e0 = KPT * tid; e0 < n_surv; e0 += KPT * T) {
          const int nv = min(KPT, n_surv - e0);
          int64_t k[KPT];
#pragma unroll
          for (int q = 0; q < KPT; q++) k[q] = load1(kbase, kdt, r0 + surv[q < nv ? e0 + q : e0]);
          hashk(k, nv);
        }
        __syncthreads();  // surv is rewritten by the next tile
      } else {
        my_surv += rows_in_tile;
        for (int e0 = KPT * tid; e0 < rows_in_tile; e0 += KPT * T) {
          const int nv = min(KPT, rows_in_tile - e0);
          int64_t k[KPT];
          if (vec && nv == KPT) {  // r0 and e0 multiples of KPT: aligned vector loads
            if (kdt == CMP_I64) {
              const longlong2* p = reinterpret_cast<const longlong2*>(reinterpret_cast<const long long*>(kbase) + r0 + e0);
#pragma unroll
              for (int q = 0; q < KPT / 2; q++) {
                const longlong2 u = __ldg(p + q);
                k[2 * q] = u.x, k[2 * q + 1] = u.y;
              }
            } else {
              const int2* p = reinterpret_cast<const int2*>(reinterpret_cast<const int32_t*>(kbase) + r0 + e0);
#pragma unroll
              for (int q = 0; q < KPT / 2; q++) {
                const int2 u = __ldg(p + q);
                k[2 * q] = u.x, k[2 * q + 1] = u.y;
              }
            }
          } else {
#pragma unroll
            for (int q = 0; q < KPT; q++) k[q] = load1(kbase, kdt, r0 + e0 + (q < nv ? q : 0));
          }
          hashk(k, nv);
        }
      }
    }
    if (it.count_surv && tid == 0 && my_surv)
      atomicAdd(reinterpret_cast<unsigned long long*>(tb->survivors), (unsigned long long)my_surv);
  }
  if (cur >= 0) flush();
  // Launched as a programmatic dependent of the counting pass (when the build has one):
  // finish only after it has, so that the build's later launches on the stream, which
  // wait for this grid, also find the counting pass complete.  Without a primary this
  // returns at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <bool PK, bool P2>
static cudaError_t launch_uniq_t(const BuildArgs& a, int32_t grid, int32_t threads, int32_t tile_rows, cudaStream_t st) {
  auto k = k_uniq_hash<PK, P2>;
  const size_t smem = uniq_smem_bytes(a.u_words, tile_rows);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  BuildArgs b = a;
  b.tile_rows = tile_rows;
  b.m31 = 1u << 31;
  b.m4 = 4;
  // programmatic dependent launch: may start while the previous kernel on the stream runs,
  // once that kernel allows it (the counting pass does, at its start)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(threads));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, b);
}

cudaError_t launch_uniq(const BuildArgs& a, int32_t grid, int32_t threads, int32_t tile_rows, cudaStream_t st) {
  if (a.n_uitems <= 0 || grid <= 0) return cudaSuccess;
  const bool pow2 = (a.w & (a.w - 1)) == 0;
  if (a.u_pack16) return pow2 ? launch_uniq_t<true, true>(a, grid, threads, tile_rows, st)
                              : launch_uniq_t<true, false>(a, grid, threads, tile_rows, st);
  return pow2 ? launch_uniq_t<false, true>(a, grid, threads, tile_rows, st)
              : launch_uniq_t<false, false>(a, grid, threads, tile_rows, st);
}

}  // namespace cmpk
