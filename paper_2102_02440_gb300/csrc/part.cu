// Partitioned Fast-AGMS sketches (Sec. 4.1, sketch partitioning): the build of a table's
// k-axis tensor and the exact contraction of a tree-shaped join's tensors.
//
// Build: one kernel per table.  A CTA walks tiles of the table's rows with the pushed-down
// predicate pass (tile.cuh); every survivor then evaluates, for each sketch row of the CTA's
// row group, the CW bucket and sign of each of its key columns and adds the product of the
// signs at the row-major index of the buckets.  Mode 1 privatises the group's tensors in
// shared memory (flushed with one global atomic per nonzero counter); mode 2 adds into the
// global counters, every CTA walking the row groups in the same order so that the group's
// tensors stay resident in L2.  No inter-CTA waits.
//
// Estimate: the tree is contracted one edge at a time, one launch per edge.  A launch
// contracts axis w of a [d][A][w][B] tensor (int32 counters or an int128 intermediate) with
// a [d][w] message (int32 or int128) into [d][A][B] int128 values.  B == 1: a team (a warp,
// or a CTA when there are few outputs) per output streams a contiguous row; B > 1: a CTA per
// 32 adjacent outputs, the lanes on the outputs (coalesced) and the warps splitting w.
// Sums are exact: an int128 plus a count of 2^128 wraps, which is order-independent; each
// product is range-checked.  A finalize launch takes the median.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "est_arith.cuh"
#include "tile.cuh"

namespace cmpk {

struct PartBuildArgs {
  DevTable tb;                 // axes = tb.key_col / tb.edge_id [0, k)
  const cmp_hash* hash;        // [n_edges * d]
  int64_t size;                // counters per sketch row
  uint32_t width[CMP_PART_MAX_AXES];
  uint32_t stride[CMP_PART_MAX_AXES];
  int32_t d, k;
  int32_t rows_per_group, n_groups, ctas_per_group;
  int32_t tile_rows;
};

struct PartStep {
  const void* x;   // [d][A][w][B]: int32 (x_wide 0) or int128
  const void* v;   // [d][w]: int32 (v_wide 0) or int128
  i128* y;         // [d][A][B]
  int64_t A, B, x_rs, v_rs;  // x_rs, v_rs: entries between consecutive sketch rows
  int32_t w, d;
  int32_t vec;     // int32 x and v, w, x_rs, v_rs multiples of 4 and 16-byte aligned rows
  uint32_t* oor;   // [d] out-of-range flags
  int32_t* status; // device status word (a bounded wait that ran out)
  uint32_t wait_polls;  // bulk kernel: polls of each chunk's wait before it gives up
};

namespace {

// ------------------------------------------------------------------ build
template <int K>
__host__ __device__ constexpr int axes_or_1() { return K > 0 ? K : 1; }

size_t part_build_smem(int rpg, int k, int R, int64_t size, bool private_ctr) {
  size_t b = align16(size_t(rpg) * size_t(std::max(k, 1)) * sizeof(PairParam)) + align16(size_t(R) * 2) + 16;
  if (private_ctr) b += size_t(rpg) * size_t(size) * 4;
  return b;
}

template <int K, bool SMEM, bool POW2>
__global__ void __launch_bounds__(1024) k_part_build(const __grid_constant__ PartBuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, T = blockDim.x;
  const int R = A.tile_rows, rpg = A.rows_per_group;
  PairParam* prm = reinterpret_cast<PairParam*>(smem);
  uint16_t* surv = reinterpret_cast<uint16_t*>(smem + align16(size_t(rpg) * axes_or_1<K>() * sizeof(PairParam)));
  int32_t* sint = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(surv) + align16(size_t(R) * 2));
  int32_t* ctr = sint + 4;  // mode 1: [rpg][size]
  const DevTable& tb = A.tb;
  const int64_t n_rows = tb.n_rows;
  const int64_t n_tiles = (n_rows + R - 1) / R;
  const bool vec = tb.vec_ok != 0;
  const bool filtered = tb.filtered != 0;
  int g0, g1, c, C;
  if (SMEM) {
    g0 = blockIdx.x / A.ctas_per_group;
    g1 = g0 + 1;
    c = blockIdx.x % A.ctas_per_group;
    C = A.ctas_per_group;
  } else {
    g0 = 0;
    g1 = A.n_groups;
    c = blockIdx.x;
    C = gridDim.x;
  }
  const void* kcol[axes_or_1<K>()];
  int32_t kdt[axes_or_1<K>()];
#pragma unroll
  for (int l = 0; l < K; l++) {
    kcol[l] = tb.col[tb.key_col[l]];
    kdt[l] = tb.dtype[tb.key_col[l]];
  }
  int64_t counted = 0;
  for (int g = g0; g < g1; g++) {
    const int r_lo = g * rpg;
    const int r_n = min(rpg, A.d - r_lo);
    __syncthreads();  // the previous group's readers of prm / ctr are done
    for (int q = tid; q < r_n * K; q += T) {
      const int i = q / axes_or_1<K>(), l = q % axes_or_1<K>();
      prm[q] = make_pair_param(A.hash[int64_t(tb.edge_id[l]) * A.d + r_lo + i]);
    }
    if (SMEM)
      for (int64_t q = tid; q < int64_t(r_n) * A.size; q += T) ctr[q] = 0;
    __syncthreads();
    int32_t* out = SMEM ? ctr : tb.counters + int64_t(r_lo) * A.size;
    for (int64_t tile = c; tile < n_tiles; tile += C) {
      const int64_t r0 = tile * R;
      const int rows_in_tile = int(n_rows - r0 < R ? n_rows - r0 : int64_t(R));
      const int n_surv = tile_survivors(&tb, r0, rows_in_tile, R, vec, surv, sint);
      if (g == 0 && tid == 0) counted += n_surv;
      if (K == 0) {
        if (tid < r_n && n_surv) atomicAdd(out + int64_t(tid) * A.size, n_surv);
      } else {
        for (int s = tid; s < n_surv; s += T) {
          const int64_t row = r0 + (filtered ? int64_t(surv[s]) : int64_t(s));
          KeyPow kp[axes_or_1<K>()];
          bool small = true;
#pragma unroll
          for (int l = 0; l < K; l++) {
            const uint64_t x = key_field(load1(kcol[l], kdt[l], row));
            kp[l] = key_powers(x);
            small = small && x < (1ull << 31);
          }
          auto update = [&](auto smallx) {
            constexpr bool SX = decltype(smallx)::value;
            for (int i = 0; i < r_n; i++) {
              uint32_t idx = 0;
              int sg = 1;
#pragma unroll
              for (int l = 0; l < K; l++) {
                const PairParam& q = prm[i * K + l];
                idx += cw_bucket<POW2, SX>(q, kp[l], A.width[l]) * A.stride[l];
                sg *= cw_sign<SX>(q, kp[l]);
              }
              atomicAdd(out + int64_t(i) * A.size + idx, sg);
            }
          };
          if (__all_sync(__activemask(), small)) update(std::true_type{});
          else update(std::false_type{});
        }
      }
      __syncthreads();  // surv is rewritten by the next tile
    }
    if (SMEM) {
      __syncthreads();
      int32_t* gout = tb.counters + int64_t(r_lo) * A.size;
      for (int64_t q = tid; q < int64_t(r_n) * A.size; q += T) {
        const int32_t v = ctr[q];
        if (v) atomicAdd(gout + q, v);
      }
    }
  }
  if (tid == 0 && counted)
    atomicAdd(reinterpret_cast<unsigned long long*>(tb.survivors), static_cast<unsigned long long>(counted));
}

template <int K, bool SMEM, bool POW2>
cudaError_t launch_part_build_t(const PartBuildArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  auto kern = k_part_build<K, SMEM, POW2>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_part_build_k(const PartBuildArgs& a, bool smem_mode, bool pow2, int grid, int threads,
                                size_t smem, cudaStream_t st) {
  if (smem_mode)
    return pow2 ? launch_part_build_t<K, true, true>(a, grid, threads, smem, st)
                : launch_part_build_t<K, true, false>(a, grid, threads, smem, st);
  return pow2 ? launch_part_build_t<K, false, true>(a, grid, threads, smem, st)
              : launch_part_build_t<K, false, false>(a, grid, threads, smem, st);
}

// ------------------------------------------------------------ contraction
__device__ __forceinline__ int32_t ld(const int32_t* p) { return __ldg(p); }
__device__ __forceinline__ i128 ld(const i128* p) {
  const longlong2 q = __ldg(reinterpret_cast<const longlong2*>(p));
  return (i128(q.y) << 64) | i128(uint64_t(q.x));
}

// one product, true when it left int128
__device__ __forceinline__ bool pmul(int32_t x, int32_t v, i128* p) {
  *p = i128(int64_t(x) * int64_t(v));
  return false;
}
__device__ __forceinline__ bool pmul(i128 x, int32_t v, i128* p) { return mul_ovf_64(x, int64_t(v), p); }
__device__ __forceinline__ bool pmul(int32_t x, i128 v, i128* p) { return mul_ovf_64(v, int64_t(x), p); }
__device__ __forceinline__ bool pmul(i128 x, i128 v, i128* p) { return mul_ovf(x, v, p); }

// exact sum: value = s + wraps * 2^128; bad: a product left int128
struct __align__(16) Acc {
  i128 s;
  int64_t wraps;
  int32_t bad, pad;
};

__device__ __forceinline__ void acc_add(Acc& a, i128 x) {
  i128 r;
  if (add_ovf(a.s, x, &r)) a.wraps += x < 0 ? -1 : 1;
  a.s = r;
}
__device__ __forceinline__ void acc_merge(Acc& a, const Acc& b) {
  acc_add(a, b.s);
  a.wraps += b.wraps;
  a.bad |= b.bad;
}
__device__ __forceinline__ Acc acc_shfl_down(const Acc& a, int off) {
  Acc b;
  const int64_t lo = __shfl_down_sync(0xffffffffu, int64_t(a.s), off);
  const int64_t hi = __shfl_down_sync(0xffffffffu, int64_t(a.s >> 64), off);
  b.s = (i128(hi) << 64) | i128(uint64_t(lo));
  b.wraps = __shfl_down_sync(0xffffffffu, a.wraps, off);
  b.bad = __shfl_down_sync(0xffffffffu, a.bad, off);
  b.pad = 0;
  return b;
}
__device__ __forceinline__ Acc warp_sum(Acc a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const Acc b = acc_shfl_down(a, off);
    if ((threadIdx.x & 31) + off < 32) acc_merge(a, b);
  }
  return a;
}

__device__ __forceinline__ void store_out(const PartStep& S, int64_t i, int64_t o, const Acc& a) {
  S.y[i * S.A * S.B + o] = a.s;
  if (a.bad || a.wraps) atomicOr(S.oor + i, 1u);
}

constexpr int kContractThreads = 256;

// B == 1: out[i][a] = sum_j x[i][a][j] v[i][j]; one team of G threads per output.
template <typename TX, typename TV, int G>
__global__ void __launch_bounds__(kContractThreads) k_part_dot(const __grid_constant__ PartStep S) {
  constexpr int TEAMS = kContractThreads / G;
  constexpr bool NARROW = std::is_same<TX, int32_t>::value && std::is_same<TV, int32_t>::value;
  __shared__ Acc red[kContractThreads / 32];
  const int lane = threadIdx.x % G, team = threadIdx.x / G;
  const int64_t items = int64_t(S.d) * S.A;
  const TX* X = static_cast<const TX*>(S.x);
  const TV* V = static_cast<const TV*>(S.v);
  for (int64_t item = int64_t(blockIdx.x) * TEAMS + team; item < items; item += int64_t(gridDim.x) * TEAMS) {
    const int64_t i = item / S.A, a = item % S.A;
    const TX* xr = X + i * S.x_rs + a * S.w;
    const TV* vr = V + i * S.v_rs;
    Acc acc{0, 0, 0, 0};
    if constexpr (NARROW) {
      // |product| <= 2^62 and w <= 2^20 terms: the int128 sum cannot wrap
      i128 s0 = 0, s1 = 0;
      if (S.vec) {
        const int4* x4 = reinterpret_cast<const int4*>(xr);
        const int4* v4 = reinterpret_cast<const int4*>(vr);
        const int n4 = S.w >> 2;
        int j = lane;
        for (; j + 3 * G < n4; j += 4 * G) {  // four independent 16-byte loads in flight per lane
          const int4 p0 = __ldg(x4 + j), p1 = __ldg(x4 + j + G), p2 = __ldg(x4 + j + 2 * G), p3 = __ldg(x4 + j + 3 * G);
          const int4 q0 = __ldg(v4 + j), q1 = __ldg(v4 + j + G), q2 = __ldg(v4 + j + 2 * G), q3 = __ldg(v4 + j + 3 * G);
          s0 += i128(int64_t(p0.x) * q0.x) + i128(int64_t(p0.y) * q0.y);
          s1 += i128(int64_t(p0.z) * q0.z) + i128(int64_t(p0.w) * q0.w);
          s0 += i128(int64_t(p1.x) * q1.x) + i128(int64_t(p1.y) * q1.y);
          s1 += i128(int64_t(p1.z) * q1.z) + i128(int64_t(p1.w) * q1.w);
          s0 += i128(int64_t(p2.x) * q2.x) + i128(int64_t(p2.y) * q2.y);
          s1 += i128(int64_t(p2.z) * q2.z) + i128(int64_t(p2.w) * q2.w);
          s0 += i128(int64_t(p3.x) * q3.x) + i128(int64_t(p3.y) * q3.y);
          s1 += i128(int64_t(p3.z) * q3.z) + i128(int64_t(p3.w) * q3.w);
        }
        for (; j < n4; j += G) {
          const int4 p = __ldg(x4 + j), q = __ldg(v4 + j);
          s0 += i128(int64_t(p.x) * q.x) + i128(int64_t(p.y) * q.y);
          s1 += i128(int64_t(p.z) * q.z) + i128(int64_t(p.w) * q.w);
        }
      } else {
        for (int j = lane; j < S.w; j += G) s0 += i128(int64_t(__ldg(xr + j)) * __ldg(vr + j));
      }
      acc.s = s0 + s1;
    } else {
      for (int j = lane; j < S.w; j += G) {
        i128 p;
        acc.bad |= pmul(ld(xr + j), ld(vr + j), &p) ? 1 : 0;
        acc_add(acc, p);
      }
    }
    acc = warp_sum(acc);
    if (G > 32) {
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 1; w < G / 32; w++) acc_merge(acc, red[w]);
        store_out(S, i, a, acc);
      }
      __syncthreads();
    } else if (lane == 0) {
      store_out(S, i, a, acc);
    }
  }
}

// B > 1: out[i][a][b] = sum_j x[i][a][j][b] v[i][j]; a CTA per 32 adjacent b, warps over j.
template <typename TX, typename TV>
__global__ void __launch_bounds__(kContractThreads) k_part_col(const __grid_constant__ PartStep S) {
  constexpr int NW = kContractThreads / 32;
  __shared__ Acc red[NW][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nb = (S.B + 31) / 32;
  const int64_t items = int64_t(S.d) * S.A * nb;
  const TX* X = static_cast<const TX*>(S.x);
  const TV* V = static_cast<const TV*>(S.v);
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t bb = item % nb, ia = item / nb;
    const int64_t a = ia % S.A, i = ia / S.A;
    const int64_t b = bb * 32 + lane;
    Acc acc{0, 0, 0, 0};
    if (b < S.B) {
      const TX* xc = X + i * S.x_rs + a * int64_t(S.w) * S.B + b;
      const TV* vr = V + i * S.v_rs;
#pragma unroll 4
      for (int j = warp; j < S.w; j += NW) {
        i128 p;
        acc.bad |= pmul(ld(xc + int64_t(j) * S.B), ld(vr + j), &p) ? 1 : 0;
        acc_add(acc, p);
      }
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
      for (int w = 1; w < NW; w++) acc_merge(acc, red[w][lane]);
      if (b < S.B) store_out(S, i, a * S.B + b, acc);
    }
    __syncthreads();
  }
}

// ---- B == 1 with int32 rows streamed through shared memory by the bulk-copy engine.
// Each warp owns a contiguous run of outputs (rows of x) and a ring of kBulkStages
// buffers of kBulkChunk bytes: lane 0 starts the asynchronous copy of each chunk
// (cp.async.bulk, completion counted in bytes on the buffer's mbarrier), the warp waits for
// the chunk, multiplies it with the message (read through L1) and lets lane 0 refill the
// buffer with the chunk kBulkStages ahead.  Every wait is bounded: when one runs out the
// warp records CMP_ETIMEOUT, waits (bounded) for its copies still in flight and returns.
constexpr int kBulkWarps = 16;
constexpr int kBulkStages = 3;
constexpr int kBulkChunk = 4096;  // bytes: 1024 int32
constexpr int64_t kBulkSmem = int64_t(kBulkWarps) * kBulkStages * kBulkChunk + kBulkWarps * kBulkStages * 8;
constexpr uint32_t kBulkWaitLimit = 1u << 22;  // try_wait polls per chunk before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// every lane polls, at most `limit` times; true once every lane has seen the phase complete
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, uint32_t limit) {
  bool done = false;
  for (uint32_t it = 0; it < limit && !done; it++) done = mbar_try_wait(bar, parity);
  return __all_sync(0xffffffffu, done);
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__global__ void __launch_bounds__(kBulkWarps * 32) k_part_dot_bulk(const __grid_constant__ PartStep S) {
  extern __shared__ __align__(128) unsigned char bulk_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* buf = bulk_smem + size_t(warp) * kBulkStages * kBulkChunk;
  uint64_t* bar = reinterpret_cast<uint64_t*>(bulk_smem + size_t(kBulkWarps) * kBulkStages * kBulkChunk) +
                  warp * kBulkStages;
  if (lane == 0) {
    for (int st = 0; st < kBulkStages; st++) mbar_init(bar + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int64_t total = int64_t(S.d) * S.A;
  const int64_t W = int64_t(gridDim.x) * kBulkWarps;
  const int64_t per = (total + W - 1) / W;
  const int64_t it0 = min(total, (int64_t(blockIdx.x) * kBulkWarps + warp) * per), it1 = min(total, it0 + per);
  const int64_t row_bytes = int64_t(S.w) * 4;  // a multiple of 16 (vec)
  const int64_t nch = (row_bytes + kBulkChunk - 1) / kBulkChunk;
  const int64_t K = (it1 - it0) * nch;
  const int32_t* X = static_cast<const int32_t*>(S.x);
  const int32_t* V = static_cast<const int32_t*>(S.v);
  auto chunk_bytes = [&](int64_t c) { return uint32_t(min(int64_t(kBulkChunk), row_bytes - c * kBulkChunk)); };
  // Positions are advanced incrementally (no 64-bit divisions per chunk): the issue cursor
  // (lane 0) runs kBulkStages chunks ahead of the consume cursor.
  struct Cursor {
    int64_t i, a, c;  // sketch row, output within it, chunk within the output's row
  };
  auto advance = [&](Cursor& u) {
    if (++u.c == nch) {
      u.c = 0;
      if (++u.a == S.A) {
        u.a = 0;
        u.i++;
      }
    }
  };
  const Cursor start{it0 / S.A, it0 % S.A, 0};
  Cursor iss = start;
  auto issue = [&](int64_t k) {  // lane 0: chunk k (at the issue cursor) into buffer k % kBulkStages
    const int32_t* src = X + iss.i * S.x_rs + iss.a * S.w + iss.c * (kBulkChunk / 4);
    const int st = int(k % kBulkStages);
    const uint32_t bytes = chunk_bytes(iss.c);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the generic reads of the buffer
    mbar_expect_tx(bar + st, bytes);
    bulk_copy_g2s(buf + size_t(st) * kBulkChunk, src, bytes, bar + st);
    advance(iss);
  };
  if (lane == 0)
    for (int64_t k = 0; k < min(K, int64_t(kBulkStages)); k++) issue(k);
  // |product| <= 2^62 and w <= 2^20 terms: the int128 sum cannot wrap
  i128 s0 = 0, s1 = 0;
  Cursor cur = start;
  int st = 0;
  uint32_t parity = 0;
  for (int64_t k = 0; k < K; k++) {
    if (!mbar_wait_warp(bar + st, parity, S.wait_polls)) {
      if (lane == 0) set_status(S.status, CMP_ETIMEOUT);
      // the copies still in flight, each waited for with the full bound, so that none is
      // left writing this CTA's shared memory after it exits
      for (int64_t kk = k; kk < min(K, k + kBulkStages); kk++)
        mbar_wait_warp(bar + int(kk % kBulkStages), uint32_t((kk / kBulkStages) & 1), kBulkWaitLimit);
      return;
    }
    const int n4 = int(chunk_bytes(cur.c) / 16);
    const int4* xs = reinterpret_cast<const int4*>(buf + size_t(st) * kBulkChunk);
    const int4* vs = reinterpret_cast<const int4*>(V + cur.i * S.v_rs + cur.c * (kBulkChunk / 4));
    for (int j = lane; j < n4; j += 32) {
      const int4 p = xs[j], q = __ldg(vs + j);
      s0 += i128(int64_t(p.x) * q.x) + i128(int64_t(p.y) * q.y);
      s1 += i128(int64_t(p.z) * q.z) + i128(int64_t(p.w) * q.w);
    }
    __syncwarp();  // every lane is done with the buffer
    if (lane == 0 && k + kBulkStages < K) issue(k + kBulkStages);
    if (cur.c == nch - 1) {  // the output's row is complete
      Acc acc{s0 + s1, 0, 0, 0};
      acc = warp_sum(acc);
      if (lane == 0) S.y[cur.i * S.A + cur.a] = acc.s;  // B == 1
      s0 = s1 = 0;
    }
    advance(cur);
    if (++st == kBulkStages) {
      st = 0;
      parity ^= 1u;
    }
  }
}

template <typename TX, typename TV>
cudaError_t launch_step_t(const PartStep& S, int sms, cudaStream_t st) {
  if (S.B == 1) {
    const int64_t items = int64_t(S.d) * S.A;
    if (std::is_same<TX, int32_t>::value && std::is_same<TV, int32_t>::value && S.vec && S.w >= 1024 &&
        items >= int64_t(sms) * kBulkWarps) {  // long int32 rows, enough of them: stream them in bulk
      cudaError_t e = cudaFuncSetAttribute(k_part_dot_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kBulkSmem));
      if (e != cudaSuccess) return e;
      const int64_t grid = std::min<int64_t>((items + kBulkWarps - 1) / kBulkWarps, int64_t(sms));
      k_part_dot_bulk<<<unsigned(grid), kBulkWarps * 32, size_t(kBulkSmem), st>>>(S);
    } else if (items >= int64_t(2) * sms * 8 || S.w < 1024) {
      const int64_t grid = std::min<int64_t>((items + 7) / 8, int64_t(sms) * 8);
      k_part_dot<TX, TV, 32><<<unsigned(grid), kContractThreads, 0, st>>>(S);
    } else {
      const int64_t grid = std::min<int64_t>(items, int64_t(sms) * 8);
      k_part_dot<TX, TV, kContractThreads><<<unsigned(grid), kContractThreads, 0, st>>>(S);
    }
  } else {
    const int64_t items = int64_t(S.d) * S.A * ((S.B + 31) / 32);
    const int64_t grid = std::min<int64_t>(items, int64_t(sms) * 8);
    k_part_col<TX, TV><<<unsigned(grid), kContractThreads, 0, st>>>(S);
  }
  return cudaGetLastError();
}

cudaError_t launch_step(const PartStep& S, bool x_wide, bool v_wide, int sms, cudaStream_t st) {
  if (!x_wide && !v_wide) return launch_step_t<int32_t, int32_t>(S, sms, st);
  if (!x_wide) return launch_step_t<int32_t, i128>(S, sms, st);
  if (!v_wide) return launch_step_t<i128, int32_t>(S, sms, st);
  return launch_step_t<i128, i128>(S, sms, st);
}

__global__ void __launch_bounds__(64) k_part_finalize(const void* root, int32_t root_wide, int64_t root_rs,
                                                      const uint32_t* __restrict__ oor, int32_t d,
                                                      double scale, double* __restrict__ est,
                                                      int64_t* __restrict__ row_est, int32_t* status) {
  __shared__ i128 rows[CMP_MAX_D];
  __shared__ int32_t any_oor;
  const int i = threadIdx.x;
  if (i == 0) any_oor = 0;
  __syncthreads();
  if (i < d) {
    const i128 v = root_wide ? ld(static_cast<const i128*>(root) + i * root_rs)
                             : i128(ld(static_cast<const int32_t*>(root) + i * root_rs));
    rows[i] = v;
    if (row_est) {
      row_est[2 * i] = int64_t(uint64_t(u128(v)));
      row_est[2 * i + 1] = int64_t(uint64_t(u128(v) >> 64));
    }
    if (oor[i]) atomicOr(&any_oor, 1);
  }
  __syncthreads();
  if (i != 0) return;
  if (any_oor) {
    *est = __longlong_as_double(0x7ff8000000000000ll);
    set_status(status, CMP_EOVERFLOW);
    return;
  }
  for (int a = 1; a < d; a++) {  // insertion sort of exact integers
    const i128 v = rows[a];
    int b = a - 1;
    while (b >= 0 && rows[b] > v) {
      rows[b + 1] = rows[b];
      b--;
    }
    rows[b + 1] = v;
  }
  const double med = (d & 1) ? i128_to_double(rows[d / 2]) : mean2_to_double(rows[d / 2 - 1], rows[d / 2]);
  *est = __dmul_rn(med, scale);  // sampled tables: one rounded product (scale 1 is exact)
}

// ------------------------------------------------------------ host plan
size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// A value of the contraction: a table's tensor (int32) or an intermediate in the workspace.
struct Val {
  int32_t table;     // >= 0: the table's tensor; -1: workspace
  int64_t off;       // workspace byte offset (int128 entries)
  int64_t rs;        // entries per sketch row
};

struct PStep {
  Val x, v;
  int64_t y_off, A, B;
  int32_t w;
};

struct PartPlan {
  std::vector<PStep> steps;
  Val root;
  size_t ws_bytes;
};

cmp_status check_join(const cmp_part_join* j, int32_t d, std::vector<int32_t>* axis_begin) {
  if (!j || d < 1 || d > CMP_MAX_D) return CMP_EINVAL;
  const int nt = j->n_tables, ne = j->n_edges;
  if (nt < 1 || nt > CMP_MAX_TABLES || ne != nt - 1 || !j->n_axes || !j->tensor) return CMP_EINVAL;
  if (j->sample_rate)
    for (int t = 0; t < nt; t++)
      if (!(j->sample_rate[t] >= 0.0 && j->sample_rate[t] <= 1.0)) return CMP_EINVAL;  // NaN fails too
  if (ne > 0 && (!j->edge_u || !j->edge_v || !j->width || !j->axis_edge)) return CMP_EINVAL;
  for (int e = 0; e < ne; e++) {
    const int u = j->edge_u[e], v = j->edge_v[e];
    if (u < 0 || u >= nt || v < 0 || v >= nt || u == v) return CMP_EINVAL;
    if (j->width[e] < 1 || j->width[e] > CMP_MAX_W) return CMP_EINVAL;
  }
  axis_begin->assign(nt + 1, 0);
  for (int t = 0; t < nt; t++) {
    const int k = j->n_axes[t];
    if (k < 0 || k > CMP_PART_MAX_AXES || !j->tensor[t]) return CMP_EINVAL;
    (*axis_begin)[t + 1] = (*axis_begin)[t] + k;
  }
  if ((*axis_begin)[nt] != 2 * ne) return CMP_EINVAL;
  for (int t = 0; t < nt; t++) {
    int64_t size = 1;
    for (int q = (*axis_begin)[t]; q < (*axis_begin)[t + 1]; q++) {
      const int e = j->axis_edge[q];
      if (e < 0 || e >= ne || (j->edge_u[e] != t && j->edge_v[e] != t)) return CMP_EINVAL;
      for (int r = (*axis_begin)[t]; r < q; r++)
        if (j->axis_edge[r] == e) return CMP_EINVAL;
      size *= j->width[e];
      if (size > CMP_PART_MAX_SIZE) return CMP_EINVAL;
    }
  }
  // every edge appears at both endpoints (2 ne axes in total, each an incident edge, no
  // repeats): now check the tree is connected
  std::vector<int> seen(nt, 0), stack{0};
  seen[0] = 1;
  int reached = 1;
  while (!stack.empty()) {
    const int t = stack.back();
    stack.pop_back();
    for (int e = 0; e < ne; e++) {
      if (j->edge_u[e] != t && j->edge_v[e] != t) continue;
      const int o = j->edge_u[e] == t ? j->edge_v[e] : j->edge_u[e];
      if (!seen[o]) {
        seen[o] = 1;
        reached++;
        stack.push_back(o);
      }
    }
  }
  return reached == nt ? CMP_OK : CMP_EINVAL;
}

// message of table t toward parent_edge (-1 at the root), steps appended in order
Val plan_message(const cmp_part_join* j, int32_t d, const std::vector<int32_t>& ab, int t, int parent_edge,
                 PartPlan* P, size_t* off) {
  std::vector<int> axes(j->axis_edge + ab[t], j->axis_edge + ab[t + 1]);
  std::vector<int64_t> shape;
  int64_t size = 1;
  for (int e : axes) {
    shape.push_back(j->width[e]);
    size *= j->width[e];
  }
  Val cur{t, 0, size};
  for (int l = int(axes.size()) - 1; l >= 0; l--) {
    const int e = axes[l];
    if (e == parent_edge) continue;
    const int child = j->edge_u[e] == t ? j->edge_v[e] : j->edge_u[e];
    const Val v = plan_message(j, d, ab, child, e, P, off);
    PStep s;
    s.x = cur;
    s.v = v;
    s.A = 1;
    for (int m = 0; m < l; m++) s.A *= shape[m];
    s.B = 1;
    for (size_t m = l + 1; m < shape.size(); m++) s.B *= shape[m];
    s.w = int32_t(shape[l]);
    s.y_off = int64_t(*off);
    *off += al256(size_t(d) * size_t(s.A * s.B) * sizeof(i128));
    P->steps.push_back(s);
    cur = Val{-1, s.y_off, s.A * s.B};
    shape.erase(shape.begin() + l);
    axes.erase(axes.begin() + l);
  }
  return cur;
}

cmp_status make_plan(const cmp_part_join* j, int32_t d, PartPlan* P) {
  std::vector<int32_t> ab;
  const cmp_status st = check_join(j, d, &ab);
  if (st != CMP_OK) return st;
  size_t off = al256(size_t(d) * sizeof(uint32_t));  // out-of-range flags first
  P->steps.clear();
  P->root = plan_message(j, d, ab, 0, -1, P, &off);
  P->ws_bytes = off;
  return CMP_OK;
}

}  // namespace
}  // namespace cmpk

using namespace cmpk;

extern "C" {

cmp_status cmp_part_build(const cmp_table* table, int32_t d, const int32_t* width_host, const cmp_hash* hash_dev,
                          int32_t n_edges, int32_t* counters_dev, int64_t* survivors_dev,
                          const cmp_part_build_cfg* cfg, void* stream) {
  cmp_status st = check_table(table, d, 1, n_edges);
  if (st != CMP_OK) return st;
  const int k = table->n_sketches;
  if (k > CMP_PART_MAX_AXES || !counters_dev || !survivors_dev || (k && (!width_host || !hash_dev)))
    return CMP_EINVAL;
  PartBuildArgs a;
  std::memset(&a, 0, sizeof(a));
  int64_t size = 1;
  bool pow2 = true;
  for (int l = 0; l < k; l++) {
    const int32_t w = width_host[l];
    if (w < 1 || w > CMP_MAX_W) return CMP_EINVAL;
    for (int m = 0; m < l; m++)
      if (table->edge_id[m] == table->edge_id[l]) return CMP_EINVAL;
    size *= w;
    if (size > CMP_PART_MAX_SIZE) return CMP_EINVAL;
    pow2 = pow2 && (w & (w - 1)) == 0;
    a.width[l] = uint32_t(w);
  }
  for (int l = k - 1; l >= 0; l--) a.stride[l] = l == k - 1 ? 1u : a.stride[l + 1] * a.width[l + 1];
  // launch shape
  int mode = cfg ? cfg->mode : 0;
  if (mode < 0 || mode > 2) return CMP_EINVAL;
  const int threads = (cfg && cfg->threads > 0) ? cfg->threads : 1024;
  const int R = (cfg && cfg->tile_rows > 0) ? cfg->tile_rows : 4096;
  if (threads < 32 || threads > 1024 || threads % 32 || R < 128 || R > 16384 || R % 128) return CMP_EINVAL;
  if (cfg && (cfg->rows_per_cta < 0 || cfg->ctas_per_sm < 0)) return CMP_EINVAL;
  const size_t optin = smem_optin_bytes();
  const size_t row_bytes = size_t(size) * 4;
  const size_t overhead = part_build_smem(d, k, R, size, false) + 1024;
  if (mode == 0) mode = row_bytes <= 64 * 1024 && row_bytes + overhead <= optin ? 1 : 2;
  int cps = (cfg && cfg->ctas_per_sm > 0) ? cfg->ctas_per_sm : 0;
  int rpg;
  if (mode == 1) {
    if (!cps) cps = size_t(d) * row_bytes + overhead <= optin / 2 ? 2 : 1;
    const size_t per_cta = optin / size_t(cps) - (cps > 1 ? 1024 : 0);
    if (per_cta <= overhead) return CMP_EINVAL;
    rpg = int(std::min<size_t>(size_t(d), (per_cta - overhead) / row_bytes));
    if (cfg && cfg->rows_per_cta > 0) rpg = std::min(cfg->rows_per_cta, d);
    if (rpg < 1 || part_build_smem(rpg, k, R, size, true) > per_cta) return CMP_EINVAL;
  } else {
    if (!cps) cps = 2;
    // one row group's tensors in about 32 MB of L2
    rpg = int(std::max<int64_t>(1, std::min<int64_t>(d, (int64_t(32) << 20) / int64_t(row_bytes))));
    if (cfg && cfg->rows_per_cta > 0) rpg = std::min(cfg->rows_per_cta, d);
  }
  const int n_groups = (d + rpg - 1) / rpg;
  rpg = (d + n_groups - 1) / n_groups;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(counters_dev, 0, size_t(d) * row_bytes, cs) != cudaSuccess) return CMP_ECUDA;
  if (cudaMemsetAsync(survivors_dev, 0, sizeof(int64_t), cs) != cudaSuccess) return CMP_ECUDA;
  if (table->n_rows == 0) return CMP_OK;
  const int64_t n_tiles = (table->n_rows + R - 1) / R;
  const int target = sm_count() * cps;
  int grid, cpg;
  if (mode == 1) {
    cpg = int(std::max<int64_t>(1, std::min<int64_t>(n_tiles, (target + n_groups - 1) / n_groups)));
    grid = n_groups * cpg;
  } else {
    cpg = int(std::max<int64_t>(1, std::min<int64_t>(n_tiles, target)));
    grid = cpg;
  }
  a.tb = to_dev(table, counters_dev, survivors_dev);
  a.hash = hash_dev;
  a.size = size;
  a.d = d;
  a.k = k;
  a.rows_per_group = rpg;
  a.n_groups = n_groups;
  a.ctas_per_group = cpg;
  a.tile_rows = R;
  const size_t smem = part_build_smem(rpg, k, R, size, mode == 1);
  cudaError_t e;
  switch (k) {
    case 0: e = launch_part_build_k<0>(a, mode == 1, pow2, grid, threads, smem, cs); break;
    case 1: e = launch_part_build_k<1>(a, mode == 1, pow2, grid, threads, smem, cs); break;
    case 2: e = launch_part_build_k<2>(a, mode == 1, pow2, grid, threads, smem, cs); break;
    case 3: e = launch_part_build_k<3>(a, mode == 1, pow2, grid, threads, smem, cs); break;
    default: e = launch_part_build_k<4>(a, mode == 1, pow2, grid, threads, smem, cs); break;
  }
  return e == cudaSuccess ? CMP_OK : CMP_ECUDA;
}

cmp_status cmp_part_estimate_ws_bytes(const cmp_part_join* join, int32_t d, size_t* ws_bytes) {
  if (!ws_bytes) return CMP_EINVAL;
  PartPlan P;
  const cmp_status st = make_plan(join, d, &P);
  if (st != CMP_OK) return st;
  *ws_bytes = P.ws_bytes;
  return CMP_OK;
}

cmp_status cmp_part_estimate(const cmp_part_join* join, int32_t d, void* ws_dev, size_t ws_bytes, double* est_dev,
                             int64_t* row_est_dev, int32_t* status_dev, void* stream) {
  return cmp_part_estimate_ex(join, d, ws_dev, ws_bytes, est_dev, row_est_dev, status_dev, nullptr, stream);
}

cmp_status cmp_part_estimate_ex(const cmp_part_join* join, int32_t d, void* ws_dev, size_t ws_bytes, double* est_dev,
                                int64_t* row_est_dev, int32_t* status_dev, const cmp_part_estimate_cfg* cfg,
                                void* stream) {
  if (!est_dev) return CMP_EINVAL;
  if (cfg && cfg->wait_polls < -1) return CMP_EINVAL;
  const uint32_t polls = (cfg && cfg->wait_polls >= 0) ? uint32_t(cfg->wait_polls) : kBulkWaitLimit;
  PartPlan P;
  const cmp_status st = make_plan(join, d, &P);
  if (st != CMP_OK) return st;
  if (!ws_dev || ws_bytes < P.ws_bytes) return CMP_EWORKSPACE;
  if ((reinterpret_cast<uintptr_t>(ws_dev) & 255) != 0) return CMP_EINVAL;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(ws_dev);
  uint32_t* oor = reinterpret_cast<uint32_t*>(ws);
  if (cudaMemsetAsync(oor, 0, size_t(d) * sizeof(uint32_t), cs) != cudaSuccess) return CMP_ECUDA;
  auto ptr = [&](const Val& v) -> const void* {
    return v.table >= 0 ? static_cast<const void*>(join->tensor[v.table]) : static_cast<const void*>(ws + v.off);
  };
  const int sms = sm_count();
  for (const PStep& s : P.steps) {
    PartStep S;
    std::memset(&S, 0, sizeof(S));
    S.x = ptr(s.x);
    S.v = ptr(s.v);
    S.y = reinterpret_cast<i128*>(ws + s.y_off);
    S.A = s.A;
    S.B = s.B;
    S.x_rs = s.x.rs;
    S.v_rs = s.v.rs;
    S.w = s.w;
    S.d = d;
    S.oor = oor;
    S.status = status_dev;
    S.wait_polls = polls;
    const bool xw = s.x.table < 0, vw = s.v.table < 0;
    S.vec = !xw && !vw && s.w % 4 == 0 && s.x.rs % 4 == 0 && s.v.rs % 4 == 0 &&
            (reinterpret_cast<uintptr_t>(S.x) & 15) == 0 && (reinterpret_cast<uintptr_t>(S.v) & 15) == 0;
    if (launch_step(S, xw, vw, sms, cs) != cudaSuccess) return CMP_ECUDA;
  }
  double scale = 1.0;  // sampled tables: prod over the tables, ascending, of 1 / rate
  if (join->sample_rate)
    for (int t = 0; t < join->n_tables; t++) {
      const double r = join->sample_rate[t];
      if (r > 0.0 && r < 1.0) scale = scale * (1.0 / r);
    }
  k_part_finalize<<<1, 64, 0, cs>>>(ptr(P.root), P.root.table < 0 ? 1 : 0, P.root.rs, oor, d, scale, est_dev,
                                     row_est_dev, status_dev);
  return cudaGetLastError() == cudaSuccess ? CMP_OK : CMP_ECUDA;
}

}  // extern "C"
