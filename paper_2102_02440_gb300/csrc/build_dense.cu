// Presence-bitmap columns of the batched build (Sec. 3.2 "Fast-AGMS Sketches": every
// selected tuple adds xi_i(key) to bucket h_i(key) of row i).  A unique key column with a
// declared domain [base, base + cap), in a table without predicates, selects exactly the
// keys whose bit the counting pass set in the column's bitmap, once each.  Its sketch row i
// is therefore the sum over the set bits j of xi_i(base + j) at bucket h_i(base + j), and
// the keys can be visited in domain order instead of row order.
//
// In domain order the hash residues need no multiplications: for consecutive field
// elements x, x + 1, ... the bucket residue (a x + b) mod p grows by a, and the sign
// residue P(x) = (c3 x^3 + c2 x^2 + c1 x + c0) mod p follows the forward differences of a
// cubic, P(x + 1) = P(x) + D1(x), D1(x + 1) = D1(x) + D2(x), D2(x + 1) = D2(x) + D3, D3
// constant, all mod p.  Each run of kDenseRun consecutive keys evaluates P at its first
// four keys and the bucket at its first key with the products (cw_sign_residue,
// cw_bucket_residue), forms D1, D2, D3 from those values, then advances with four modular
// additions per key: the same residues as evaluating the polynomials at every key, so the
// counters are the same integers.  Key k of the domain has field element key_field(base +
// k); consecutive keys have consecutive residues (mod p), including where they cross 0.
//
// Counters: the slab's pairs in shared memory, as in the unique-key kernel (slab.cuh).
// Items: (slab, range of whole runs), clipped at run time to the runs holding the column's
// surviving keys; a CTA takes a contiguous list of items of about equal work.  A column
// the counting pass found inactive (a key outside its domain, or a key seen twice) is
// skipped here: the row kernel hashes it.  No inter-CTA waits.
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.cuh"
#include "slab.cuh"

namespace cmpk {

namespace {

constexpr int kRunWords = int(kDenseRun / 32);
constexpr int kRuns = 2;  // runs per thread in flight: independent difference chains

// Lazy residues: folded values v <= 2^61 + 3 with v = the residue (mod p).  A sum s below
// 2^64 folds, (s mod 2^61) + (s >> 61), back to <= 2^61 + 7, and below 2^63 to <= 2^61 + 3.
// D1 and D2 are folded at odd steps only (each 32-key word starts at an even step): after an
// even step both are sums of two folded values, below 2^62 + 8, so at the odd step P + D1
// stays below 2^63 and D1 + D2 below 2^63 + 16; P is folded at every step (its residue
// gives the sign).
__device__ __forceinline__ uint64_t add_lazy(uint64_t u, uint64_t v) { return fold61(u + v); }
__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b) { return a >= b ? a - b : a + kP61 - b; }

// Difference state of one (run, pair): sign residue P, its differences D1, D2, and the
// bucket residue B at the current key.
struct Diff {
  uint64_t P, D1, D2, B;
};

// The state at field element x0 (< p) for the pair's parameters; D3 is returned apart.
__device__ __forceinline__ Diff diff_at(const PairParam& q, uint64_t x0, uint64_t* D3) {
  uint64_t v[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    uint64_t x = x0 + uint64_t(j);
    x = x >= kP61 ? x - kP61 : x;
    v[j] = cw_sign_residue<false>(q, key_powers(x));
  }
  const uint64_t d01 = sub_mod(v[1], v[0]), d12 = sub_mod(v[2], v[1]), d23 = sub_mod(v[3], v[2]);
  const uint64_t e0 = sub_mod(d12, d01), e1 = sub_mod(d23, d12);
  *D3 = sub_mod(e1, e0);
  Diff s;
  s.P = v[0];
  s.D1 = d01;
  s.D2 = e0;
  s.B = cw_bucket_residue<false>(q, key_powers(x0));
  return s;
}

}  // namespace

size_t dense_smem_bytes(int32_t words) { return align16(sizeof(uint32_t) * size_t(words)); }

// THREADS: 512 alone on the SM, 256 beside a CTA of the counting pass (128 registers each)
template <bool PACK16, bool POW2, int THREADS>
__global__ void __launch_bounds__(THREADS, 512 / THREADS) k_dense_hash(const __grid_constant__ BuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PairParam prm[kUniqMaxPairs];
  __shared__ int32_t* grow[kUniqMaxPairs];
  __shared__ int32_t s_active;
  __shared__ long long s_lo, s_hi;  // domain offsets of the surviving keys: [s_lo, s_hi)
  const int tid = threadIdx.x, T = blockDim.x;
  // the first part, beside the counting pass: the second part (512 threads, one CTA per SM)
  // may take each SM as soon as both have left it
  if (A.dense_part == 1) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const uint32_t w = uint32_t(A.w);
  uint32_t* cs = reinterpret_cast<uint32_t*>(smem);
  const int words = A.d_words;
  const int64_t i_begin = A.d_cta_item[blockIdx.x], i_end = A.d_cta_item[blockIdx.x + 1];
  for (int j = tid; j < words; j += T) cs[j] = PACK16 ? kWordBias : 0u;
  int cur = -1;  // slab whose counters are in shared memory (block-uniform)
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
    const UniqItem it = A.ditem[ii];
    const UniqSlab& sl = A.dslab[it.slab];
    const int ai = sl.pad;
    const AggCol& ac = A.agg[ai];
    const DevTable* tb = A.tables + sl.table;
    if (it.slab != cur) {
      if (cur >= 0 && s_active) flush();
      __syncthreads();  // s_active is rewritten below
      if (tid < sl.n_pairs) {
        const int pair = sl.pair[tid];
        const int s = pair / A.d, i = pair % A.d;
        prm[tid] = make_pair_param(A.hash[size_t(tb->edge_id[s]) * A.d + i]);
        grow[tid] = tb->counters + size_t(pair) * w;
      }
      if (tid == 0) {
        int64_t kmin = 0, range = 0;
        s_active = agg_active(ac, ai, A.ws, &kmin, &range) ? 1 : 0;
        s_lo = (long long)(uint64_t(kmin) - uint64_t(ac.base));
        s_hi = s_lo + range;
      }
      cur = it.slab;
      n_pairs = sl.n_pairs;
      __syncthreads();
    }
    if (!s_active) continue;  // block-uniform: the row kernel hashes this column
    const int64_t lo = max(int64_t(it.row_begin), int64_t(s_lo) / kDenseRun * kDenseRun);
    const int64_t hi = min(int64_t(it.row_end), int64_t(s_hi));
    if (lo >= hi) continue;
    const int64_t n_runs = (hi - lo + kDenseRun - 1) / kDenseRun;
    const uint32_t* bm = reinterpret_cast<const uint32_t*>(A.ws + ac.off);
    const int64_t cut = (n_runs * A.dense_cut + 1023) / 1024;  // this part's runs [run_lo, run_hi)
    const int64_t run_lo = A.dense_part == 2 ? cut : 0, run_hi = A.dense_part == 1 ? cut : n_runs;
    for (int64_t r0 = run_lo + tid; r0 < run_hi; r0 += int64_t(kRuns) * T) {
      // runs r0 and r0 + T of this item (when present): bitmap words and first keys
      uint32_t wd[kRuns][kRunWords];
      uint64_t x0[kRuns];
      bool has[kRuns];
#pragma unroll
      for (int u = 0; u < kRuns; u++) {
        const int64_t r = r0 + int64_t(u) * T;
        has[u] = r < run_hi;
        const int64_t k0 = lo + r * kDenseRun;  // a multiple of kDenseRun: 32-byte aligned words
        if (has[u]) {
          const uint4* p4 = reinterpret_cast<const uint4*>(bm + k0 / 32);
          const uint4 a = __ldg(p4), b = __ldg(p4 + 1);
          wd[u][0] = a.x, wd[u][1] = a.y, wd[u][2] = a.z, wd[u][3] = a.w;
          wd[u][4] = b.x, wd[u][5] = b.y, wd[u][6] = b.z, wd[u][7] = b.w;
        } else {
#pragma unroll
          for (int q = 0; q < kRunWords; q++) wd[u][q] = 0;
        }
        x0[u] = key_field(int64_t(uint64_t(ac.base) + uint64_t(has[u] ? k0 : lo)));
      }
      for (int p = 0; p < n_pairs; p++) {
        const PairParam q = prm[p];
        const uint64_t a_step = q.a_lo | (uint64_t(q.a_hi) << 31);
        int32_t* g = grow[p];
        uint32_t* c = PACK16 ? cs : cs + size_t(p) * w;
        Diff st[kRuns];
        uint64_t D3[kRuns];
#pragma unroll
        for (int u = 0; u < kRuns; u++) st[u] = diff_at(q, x0[u], &D3[u]);
        uint32_t wq[kRuns][kRunWords];  // the words, consumed from the front
#pragma unroll
        for (int u = 0; u < kRuns; u++)
#pragma unroll
          for (int q8 = 0; q8 < kRunWords; q8++) wq[u][q8] = wd[u][q8];
#pragma unroll 1
        for (int q8 = 0; q8 < kRunWords; q8++) {
          uint32_t m[kRuns];
#pragma unroll
          for (int u = 0; u < kRuns; u++) {
            m[u] = wq[u][0];
#pragma unroll
            for (int j = 0; j + 1 < kRunWords; j++) wq[u][j] = wq[u][j + 1];  // static indices: registers
          }
#pragma unroll 4
          for (int b = 0; b < 32; b++) {
#pragma unroll
            for (int u = 0; u < kRuns; u++) {
              if (m[u] & 1u) {
                // residues: P or P - p (P <= p + 4 < 2p); its parity flips with the subtraction
                const uint32_t geP = uint32_t((st[u].P + 1) >> 61), geB = uint32_t((st[u].B + 1) >> 61);
                const int sg = 1 - 2 * int((uint32_t(st[u].P) ^ geP) & 1u);
                uint32_t h;
                if (POW2) h = (uint32_t(st[u].B) + geB) & (w - 1);  // -p = 1 (mod w)
                else h = uint32_t((geB ? st[u].B - kP61 : st[u].B) % w);
                if (PACK16) counter_add<true>(c, g, h, sg, w);
                else red_add_shared(reinterpret_cast<int32_t*>(c) + h, sg);
              }
              m[u] >>= 1;
              st[u].P = add_lazy(st[u].P, st[u].D1);
              st[u].D1 = (b & 1) ? add_lazy(st[u].D1, st[u].D2) : st[u].D1 + st[u].D2;
              st[u].D2 = (b & 1) ? add_lazy(st[u].D2, D3[u]) : st[u].D2 + D3[u];
              st[u].B = add_lazy(st[u].B, a_step);
            }
          }
        }
      }
    }
  }
  if (cur >= 0 && s_active) flush();
  // Launched as a programmatic dependent (of the hashing of the counted keys, of the second
  // launch of a split counting pass, or, the second part, of the first part): finish only
  // after it has, so that the stream's later work also finds it complete.
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <bool PK, bool P2, int TH>
static cudaError_t launch_dense_t(const BuildArgs& a, int32_t grid, bool pdl, cudaStream_t st) {
  auto k = k_dense_hash<PK, P2, TH>;
  const size_t smem = dense_smem_bytes(a.d_words);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(TH));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, a);
}

// pdl: launch as a programmatic dependent of the previous kernel on the stream, which must
// let dependents start only once every presence bitmap is complete: the hashing of the
// counted keys (it starts after the whole counting pass), or the second launch of a split
// counting pass (it starts after the first, which counts every table with a presence
// column).  Otherwise an ordinary launch.  threads: kDenseThreadsAlone or
// kDenseThreadsBeside.
cudaError_t launch_dense(const BuildArgs& a, int32_t grid, bool pdl, int32_t threads, cudaStream_t st) {
  if (a.n_ditems <= 0 || grid <= 0) return cudaSuccess;
  const bool pow2 = (a.w & (a.w - 1)) == 0;
  if (threads == kDenseThreadsBeside) {
    if (a.d_pack16)
      return pow2 ? launch_dense_t<true, true, 256>(a, grid, pdl, st) : launch_dense_t<true, false, 256>(a, grid, pdl, st);
    return pow2 ? launch_dense_t<false, true, 256>(a, grid, pdl, st) : launch_dense_t<false, false, 256>(a, grid, pdl, st);
  }
  if (a.d_pack16)
    return pow2 ? launch_dense_t<true, true, 512>(a, grid, pdl, st) : launch_dense_t<true, false, 512>(a, grid, pdl, st);
  return pow2 ? launch_dense_t<false, true, 512>(a, grid, pdl, st) : launch_dense_t<false, false, 512>(a, grid, pdl, st);
}

}  // namespace cmpk
