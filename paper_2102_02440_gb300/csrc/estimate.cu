// Sketch-merging estimate (Sec. 4.2 merge equation, iterated over a table's joins; Sec. 3.2
// inner product and median), exact in int128.
//
// Reading used for sub-plans beyond the 3-table chain of Sec. 4.1: row i of sub-plan S is
//   E_i = sum over bucket assignments j of S's edges of  prod over t in S of M_t(j|t),
// M_t the merged sketch of t (value of the sketch, among t's sketches of S's edges in
// ascending edge id, whose bucket has the minimum |.|, the first on ties).
// Evaluation: a spanning tree (BFS from the lowest table id, edges in id order) is
// contracted leaf to root; each non-tree edge index is fixed to c and summed over c.
// For a table with incoming messages m_l on its edges l != p (p = edge to its parent),
// splitting the sum by which edge attains the minimum gives threshold sums
//   G_l^>(tau) = sum_{|s_l[j]| > tau} m_l[j],  G_l^>=(tau) = sum_{|s_l[j]| >= tau} m_l[j]
// (edge l' < l loses to l iff |s_l'| > |s_l|, edge l' > l iff |s_l'| >= |s_l|):
//   out[jp] = s_p[jp] prod_{l != p} G_l^{l<p ? > : >=}(|s_p[jp]|)
//           + sum_{l != p} sum_{j : |s_l[j]| (l>p ? < : <=) |s_p[jp]|}
//                 s_l[j] m_l[j] prod_{l' != l,p} G_l'^{l'<l ? > : >=}(|s_l[j]|)
// and at the root (no p) the scalar sum_l sum_j s_l[j] m_l[j] prod_{l' != l} G_l'(...).
// With every sketch row presorted by (|C|, bucket), each G and each inner sum is a suffix
// / prefix sum read at a binary-searched rank.
#include <cuda_runtime.h>

#include "est_arith.cuh"

namespace cmpk {

// ---------------------------------------------------------------- presort
// One CTA per sketch row: keys (|C| << 32 | bucket) bitonic-sorted in shared memory.
__global__ void __launch_bounds__(1024) k_presort(const int32_t* __restrict__ C, int64_t n_rows, int32_t w,
                                                  int32_t wp2, uint32_t* __restrict__ abs_out,
                                                  int32_t* __restrict__ perm_out) {
  extern __shared__ unsigned long long key[];
  for (int64_t row = blockIdx.x; row < n_rows; row += gridDim.x) {
    const int32_t* src = C + row * w;
    for (int j = threadIdx.x; j < wp2; j += blockDim.x) {
      if (j < w) {
        const int32_t v = src[j];
        const uint32_t a = v < 0 ? uint32_t(-int64_t(v)) : uint32_t(v);
        key[j] = (static_cast<unsigned long long>(a) << 32) | uint32_t(j);
      } else {
        key[j] = ~0ull;
      }
    }
    __syncthreads();
    for (int k = 2; k <= wp2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < wp2; i += blockDim.x) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long a = key[i], b = key[ixj];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
              key[i] = b;
              key[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
      const unsigned long long kk = key[j];
      abs_out[row * w + j] = uint32_t(kk >> 32);
      perm_out[row * w + j] = int32_t(uint32_t(kk));
    }
    __syncthreads();
  }
}

// Rows longer than one shared-memory sort: chunks of kChunk keys are bitonic-sorted in
// shared memory, then runs are merged pairwise in global memory.  Each key's place in the
// merged run is its index in its own run plus the number of partner-run keys placed
// before it.
constexpr int kChunk = 8192;

// Rows of C are w long; key rows are L long (L a multiple of kChunk, keys beyond w are
// padding that sorts last).
__global__ void __launch_bounds__(1024) k_presort_chunks(const int32_t* __restrict__ C, int64_t n_rows, int32_t w,
                                                         int64_t L, unsigned long long* __restrict__ keys) {
  extern __shared__ unsigned long long key[];  // kChunk keys
  const int chunks = int(L / kChunk);
  for (int64_t blk = blockIdx.x; blk < n_rows * chunks; blk += gridDim.x) {
    const int64_t row = blk / chunks;
    const int c0 = int(blk % chunks) * kChunk;
    const int32_t* src = C + row * w;
    for (int j = threadIdx.x; j < kChunk; j += blockDim.x) {
      const int g = c0 + j;
      if (g < w) {
        const int32_t v = src[g];
        const uint32_t a = v < 0 ? uint32_t(-int64_t(v)) : uint32_t(v);
        key[j] = (static_cast<unsigned long long>(a) << 32) | uint32_t(g);
      } else {
        key[j] = ~0ull;
      }
    }
    __syncthreads();
    for (int k = 2; k <= kChunk; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < kChunk; i += blockDim.x) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long a = key[i], b = key[ixj];
            if ((a > b) == ((i & k) == 0)) {
              key[i] = b;
              key[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    unsigned long long* dst = keys + row * L + c0;
    for (int j = threadIdx.x; j < kChunk; j += blockDim.x) dst[j] = key[j];
    __syncthreads();
  }
}

// One merge level: runs of length `run` (padded row length L, a power of two times kChunk).
__global__ void k_presort_merge(const unsigned long long* __restrict__ in, unsigned long long* __restrict__ out,
                                int64_t n_rows, int64_t L, int64_t run) {
  const int64_t total = n_rows * L;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = t / L, i = t % L;
    const int64_t base = row * L + (i / (2 * run)) * (2 * run);
    const int64_t off = i % (2 * run);
    const bool left = off < run;
    const int64_t idx = left ? off : off - run;
    const unsigned long long v = in[t];
    const unsigned long long* other = in + base + (left ? run : 0);
    // partner keys placed before v: below it, and for the right run also equal to it
    // (equal keys are the padding; the left run's copies go first, so positions are a
    // permutation of the output run)
    int64_t lo = 0, hi = run;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (left ? other[mid] < v : other[mid] <= v) lo = mid + 1;
      else hi = mid;
    }
    out[base + idx + lo] = v;
  }
}

__global__ void k_presort_split(const unsigned long long* __restrict__ keys, int64_t n_rows, int32_t w, int64_t L,
                                uint32_t* __restrict__ abs_out, int32_t* __restrict__ perm_out) {
  const int64_t total = n_rows * int64_t(w);
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = t / w, j = t % w;
    const unsigned long long k = keys[row * L + j];
    abs_out[t] = uint32_t(k >> 32);
    perm_out[t] = int32_t(uint32_t(k));
  }
}

int64_t presort_padded(int32_t w) {
  int64_t L = kChunk;
  while (L < w) L <<= 1;
  return L;
}

cudaError_t launch_presort_large(const int32_t* C, int64_t n_rows, int32_t w, uint32_t* abs_out, int32_t* perm_out,
                                 void* ws, int64_t rows_per_pass, cudaStream_t st) {
  const int64_t L = presort_padded(w);
  unsigned long long* a = static_cast<unsigned long long*>(ws);
  unsigned long long* b = a + rows_per_pass * L;
  for (int64_t r0 = 0; r0 < n_rows; r0 += rows_per_pass) {
    const int64_t nr = n_rows - r0 < rows_per_pass ? n_rows - r0 : rows_per_pass;
    const int64_t nblk = nr * (L / kChunk);
    const int smem = int(sizeof(unsigned long long)) * kChunk;
    cudaError_t e = cudaFuncSetAttribute(k_presort_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_presort_chunks<<<unsigned(nblk < 4096 ? nblk : 4096), 1024, smem, st>>>(C + r0 * w, nr, w, L, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int64_t run = kChunk; run < L; run <<= 1) {
      k_presort_merge<<<4096, 256, 0, st>>>(a, b, nr, L, run);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      unsigned long long* t = a;
      a = b;
      b = t;
    }
    k_presort_split<<<4096, 256, 0, st>>>(a, nr, w, L, abs_out + r0 * w, perm_out + r0 * w);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    a = static_cast<unsigned long long*>(ws);
    b = a + rows_per_pass * L;
  }
  return cudaSuccess;
}

cudaError_t launch_presort(const int32_t* C, int64_t n_rows, int32_t w, uint32_t* abs_out, int32_t* perm_out,
                           cudaStream_t st) {
  if (n_rows <= 0) return cudaSuccess;
  int wp2 = 1;
  while (wp2 < w) wp2 <<= 1;
  const size_t smem = sizeof(unsigned long long) * size_t(wp2);
  cudaError_t e = cudaFuncSetAttribute(k_presort, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const int threads = wp2 >= 1024 ? 1024 : (wp2 < 32 ? 32 : wp2);
  const int64_t grid = n_rows < 4096 ? n_rows : 4096;
  k_presort<<<unsigned(grid), threads, smem, st>>>(C, n_rows, w, wp2, abs_out, perm_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- cross ranks
struct CrossArgs {
  const uint32_t* abs;
  const int32_t* perm;
  int32_t* ranks;
  int32_t k, d, w;
  int32_t edge[CMP_MAX_SKETCHES];
};

__device__ __forceinline__ int rank_in(const uint32_t* __restrict__ a, int w, uint32_t tau, bool strict) {
  int lo = 0, hi = w;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const uint32_t v = __ldg(a + mid);
    if (strict ? v <= tau : v < tau) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The same search in a shared-memory window (plain loads).
__device__ __forceinline__ int rank_in_shared(const uint32_t* a, int n, uint32_t tau, bool strict) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const uint32_t v = a[mid];
    if (strict ? v <= tau : v < tau) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One CTA per (x, y, row): ranks of x's sorted magnitudes in y's, or x's inverse permutation.
__global__ void k_cross_ranks(const __grid_constant__ CrossArgs A) {
  const int k = A.k, d = A.d, w = A.w;
  const int64_t blk = blockIdx.x;
  const int row = int(blk % d), y = int((blk / d) % k), x = int(blk / (int64_t(d) * k));
  int32_t* out = A.ranks + ((int64_t(x) * k + y) * d + row) * w;
  if (x == y) {
    const int32_t* perm = A.perm + (int64_t(x) * d + row) * w;
    for (int r = threadIdx.x; r < w; r += blockDim.x) out[__ldg(perm + r)] = r;
    return;
  }
  const uint32_t* ax = A.abs + (int64_t(x) * d + row) * w;
  const uint32_t* ay = A.abs + (int64_t(y) * d + row) * w;
  const bool strict = A.edge[y] < A.edge[x];
  for (int r = threadIdx.x; r < w; r += blockDim.x) out[r] = rank_in(ay, w, __ldg(ax + r), strict);
}

// Several tables per launch: table t's CTAs are [blk0[t], blk0[t + 1]), its rows start at
// row_off[t] of abs / perm and its rank block at rank_off[t] (int32 units).
constexpr int kCrossMultiTables = 16;
struct CrossMultiArgs {
  const uint32_t* abs;
  const int32_t* perm;
  int32_t* ranks;
  int32_t n, d, w;
  int64_t blk0[kCrossMultiTables + 1];
  int64_t row_off[kCrossMultiTables], rank_off[kCrossMultiTables];
  int32_t k[kCrossMultiTables];
  int32_t edge[kCrossMultiTables][CMP_MAX_SKETCHES];
};

// One CTA per (table, x, y, row, segment of kCrossSeg sorted positions of x).  x's sorted
// magnitudes are ascending, so their ranks in y's are too: the segment's ranks lie between
// the ranks of its first and last value, and that window of y's row is staged in shared
// memory (when it fits; else the searches read y's row in global memory).
constexpr int kCrossSeg = 2048;
constexpr int kCrossWin = 4096;
__global__ void __launch_bounds__(256) k_cross_ranks_multi(const __grid_constant__ CrossMultiArgs A) {
  __shared__ uint32_t win[kCrossWin];
  __shared__ int32_t s_lo, s_hi;
  const int w = A.w, d = A.d;
  const int64_t nseg = (w + kCrossSeg - 1) / kCrossSeg;
  const int64_t blk = blockIdx.x / nseg;
  const int r0 = int(blockIdx.x % nseg) * kCrossSeg, r1 = min(w, r0 + kCrossSeg);
  int t = 0;
  while (t + 1 < A.n && A.blk0[t + 1] <= blk) t++;
  const int k = A.k[t];
  const int64_t b = blk - A.blk0[t];
  const int row = int(b % d), y = int((b / d) % k), x = int(b / (int64_t(d) * k));
  int32_t* out = A.ranks + A.rank_off[t] + ((int64_t(x) * k + y) * d + row) * w;
  if (x == y) {
    const int32_t* perm = A.perm + (A.row_off[t] + int64_t(x) * d + row) * w;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) out[__ldg(perm + r)] = r;
    return;
  }
  const uint32_t* ax = A.abs + (A.row_off[t] + int64_t(x) * d + row) * w;
  const uint32_t* ay = A.abs + (A.row_off[t] + int64_t(y) * d + row) * w;
  const bool strict = A.edge[t][y] < A.edge[t][x];
  if (threadIdx.x == 0) s_lo = rank_in(ay, w, __ldg(ax + r0), strict);
  if (threadIdx.x == 32) s_hi = rank_in(ay, w, __ldg(ax + r1 - 1), strict);
  __syncthreads();
  const int lo = s_lo, n = s_hi - lo;  // block-uniform
  if (n <= kCrossWin) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) win[j] = __ldg(ay + lo + j);
    __syncthreads();
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x)
      out[r] = lo + rank_in_shared(win, n, __ldg(ax + r), strict);
  } else {
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) out[r] = rank_in(ay, w, __ldg(ax + r), strict);
  }
}

cudaError_t launch_cross_ranks_multi(const uint32_t* abs, const int32_t* perm, int32_t n_tables, const int32_t* k,
                                     const int32_t* edge_ids, int32_t d, int32_t w, int32_t* ranks, cudaStream_t st) {
  int64_t row = 0, rank = 0, e = 0;
  for (int32_t t0 = 0; t0 < n_tables; t0 += kCrossMultiTables) {
    CrossMultiArgs a;
    a.abs = abs;
    a.perm = perm;
    a.ranks = ranks;
    a.n = n_tables - t0 < kCrossMultiTables ? n_tables - t0 : kCrossMultiTables;
    a.d = d;
    a.w = w;
    int64_t blk = 0;
    for (int i = 0; i < a.n; i++) {
      const int32_t kt = k[t0 + i];
      a.blk0[i] = blk;
      a.row_off[i] = row;
      a.rank_off[i] = rank;
      a.k[i] = kt;
      for (int q = 0; q < CMP_MAX_SKETCHES; q++) a.edge[i][q] = q < kt ? edge_ids[e + q] : 0;
      blk += int64_t(kt) * kt * d;
      row += int64_t(kt) * d;
      rank += int64_t(kt) * kt * d * w;
      e += kt;
    }
    a.blk0[a.n] = blk;
    if (blk > 0) {
      k_cross_ranks_multi<<<unsigned(blk * ((w + kCrossSeg - 1) / kCrossSeg)), 256, 0, st>>>(a);
      const cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return err;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_cross_ranks(const uint32_t* abs, const int32_t* perm, int32_t k, int32_t d, int32_t w,
                               const int32_t* edge_id, int32_t* ranks, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  CrossArgs a;
  a.abs = abs;
  a.perm = perm;
  a.ranks = ranks;
  a.k = k;
  a.d = d;
  a.w = w;
  for (int i = 0; i < CMP_MAX_SKETCHES; i++) a.edge[i] = i < k ? edge_id[i] : 0;
  k_cross_ranks<<<unsigned(int64_t(k) * k * d), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- estimate helpers
namespace {

// Row `row` of the cross ranks of sketch x against sketch y of the same table.
__device__ __forceinline__ const int32_t* rank_row(const EstIn& x, const EstIn& y, int d, int row, int w) {
  return x.rk + (int64_t(y.tslot) * d + row) * w;
}

}  // namespace

// One CTA per work item (sub-plan, sketch row, range of conditioning values), persistent
// over the item list.  Per-CTA scratch in the workspace (S = int64, or int128 on retry):
//   slots [max_slots][w]  messages
//   suf   [max_suf][w+1]  suffix sums of each incoming message in its sketch's sorted
//                         order (leaf inputs: computed once per item)
//   pre   [max_in][w+1]   prefix sums of the "this edge attains the minimum" terms
// Cross ranks between the sorted rows of a table's sketches come from the cache written
// by cmp_cross_ranks (they depend on no message and no sub-plan).
// Cached subtree messages (Sec. 4.2: an (n+1)-D merge extends an n-D one; Sec. 5: merged
// sketches cached across sub-plans): a job item computes the message of one subtree over
// its connecting edge into the workspace cache, in int128; sub-plans and larger subtrees
// read it as a kInCache input.  Launch l runs [it0, it1) and reads messages of earlier
// launches only.
// A conditioned input (unit vector at c) needs no array: its threshold sum is a
// comparison with |s[c]| and its own term is one value.  When some conditioned sketch
// value s[c] is 0, every merged tensor entry at c through that table is 0 and c adds
// nothing, so it is skipped.  Products and sums are exact int128; values stored in the
// int64 arrays that do not fit flag the item for recomputation with int128 storage.
constexpr int kMaxIn = CMP_MAX_SKETCHES;
constexpr int kMaxPreChunk = 256;  // conditioning values per item whose scalars the prologue precomputes

// kIlp elements per thread have their loads issued together (memory-level parallelism);
// MAXT and MINB (resident CTAs per SM) are the launch bounds that set the register budget.
template <typename S, int kIlp, int MAXT, int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB) k_estimate_items(const __grid_constant__ EstArgs A, int retry, int64_t it0,
                                                         int64_t it1) {
  __shared__ i128 sh_i128[33];
  __shared__ int32_t sh_flag[1];
  __shared__ i128 sh_val[kMaxIn];
  __shared__ uint32_t sh_ac[kMaxIn];
  __shared__ EstOp sh_ops[kEstMaxOps];
  __shared__ EstIn sh_in[kEstMaxSubIn];
  __shared__ const int32_t* sh_cond[2 * kEstMaxCond];  // each conditioned edge's two sketches
  __shared__ int32_t sh_cond_k[2 * kEstMaxCond];       // and its ordinal
  __shared__ int32_t sh_ncond;
  // per conditioned operation (at most two per sub-plan), for every c of the chunk when
  // its other inputs are leaves: |s[c]| and the "attains the minimum" value
  __shared__ int32_t sh_pop[2], sh_pa[2];
  __shared__ uint32_t sh_cac[2][kMaxPreChunk];
  __shared__ i128 sh_cval[2][kMaxPreChunk];
  __shared__ uint8_t sh_skip[kMaxPreChunk];
  BlockScratch bs{sh_i128, sh_flag};
  const int w = A.w;
  const int64_t W1 = int64_t(w) + 1;
  unsigned char* cta = reinterpret_cast<unsigned char*>(A.scratch) + int64_t(blockIdx.x) * A.scratch_per_cta;
  S* slots = reinterpret_cast<S*>(cta);
  S* suf = slots + int64_t(A.max_slots) * w;
  S* pre = suf + int64_t(A.max_suf) * W1;
  const int tid = threadIdx.x, T = blockDim.x;

  for (int64_t it = it0 + blockIdx.x; it < it1; it += gridDim.x) {
    if (retry && A.partial_ovf[it] != 2) continue;  // block-uniform
    const EstItem item = A.items[it];
    const EstSub sb = A.subs[item.sub];
    const int64_t ro = int64_t(item.row) * w;  // row offset inside every [d][w] array
    i128* const gout = sb.job >= 0 ? A.cache + (int64_t(sb.job) * A.d + item.row) * w : nullptr;
    const int in0 = A.ops[sb.op_begin].in_begin;
    const int n_in = sb.n_ops ? A.ops[sb.op_begin + sb.n_ops - 1].in_begin + A.ops[sb.op_begin + sb.n_ops - 1].k - in0
                              : 0;
    for (int o = tid; o < sb.n_ops; o += T) {
      EstOp op = A.ops[sb.op_begin + o];
      op.in_begin -= in0;  // index into sh_in
      sh_ops[o] = op;
    }
    for (int q = tid; q < n_in; q += T) sh_in[q] = A.inputs[in0 + q];
    if (tid == 0) sh_flag[0] = 0;
    __syncthreads();
    if (tid == 0) {
      // a cached input that left int128 makes this row's result leave it too
      for (int q = 0; q < n_in; q++)
        if (sh_in[q].kind == kInCache && A.cache_ovf[int64_t(sh_in[q].slot) * A.d + item.row]) sh_flag[0] |= 1;
      int nc = 0;
      for (int q = 0; q < n_in && nc < 2 * kEstMaxCond; q++)
        if (sh_in[q].kind == kInCond) {
          sh_cond[nc] = sh_in[q].s + ro;
          sh_cond_k[nc++] = sh_in[q].slot;
        }
      sh_ncond = nc;
      // operations with one conditioned input whose other inputs are all leaves: precomputable per c
      int np = 0;
      for (int o = 0; o < sb.n_ops && np < 2; o++) {
        const EstOp& op = sh_ops[o];
        int ca = -1, n_ca = 0;
        bool leaves = true;
        for (int a = 0, l = 0; l < op.k; l++) {
          if (l == op.p) continue;
          const int kind = sh_in[op.in_begin + l].kind;
          if (kind == kInCond) {
            ca = a;
            n_ca++;
          } else {
            leaves &= kind == kInLeaf;
          }
          a++;
        }
        if (n_ca == 1 && leaves) {
          sh_pop[np] = o;
          sh_pa[np] = ca;
          np++;
        }
      }
      for (int q = np; q < 2; q++) sh_pop[q] = -1;
    }

    // ---------------- prologue: cross ranks and leaf suffix sums (independent of c)
    for (int o = 0; o < sb.n_ops; o++) {
      const EstOp op = sh_ops[o];
      const EstIn* in = sh_in + op.in_begin;
      const int p = op.p;
      const int m = op.k - (p >= 0 ? 1 : 0);
      for (int a = 0; a < m; a++) {
        const int la = a + (p >= 0 && a >= p ? 1 : 0);
        const EstIn& x = in[la];
        if (x.kind != kInLeaf) continue;
        S* sl = suf + int64_t(x.suf) * W1;
        const int32_t* perm = x.perm + ro;
        for (int r = tid; r < w; r += T) sl[r] = S(__ldg(x.msk + ro + __ldg(perm + r)));
        if (tid == 0) sl[w] = 0;
        __syncthreads();
        block_scan(sl, w, /*reverse=*/true, bs);
      }
    }
    __syncthreads();
    const int nchunk = item.c1 - item.c0;
    const bool pre_ok = sb.cond && nchunk <= kMaxPreChunk;
    if (pre_ok) {
      for (int c = item.c0 + tid; c < item.c1; c += T) {
        bool zero = false;
        for (int q = 0; q < sh_ncond; q++) zero |= __ldg(sh_cond[q] + cond_digit(c, sh_cond_k[q], w)) == 0;
        sh_skip[c - item.c0] = zero;
      }
      for (int t = tid; t < 2 * nchunk; t += T) {
        const int k = t / nchunk, c = item.c0 + t % nchunk;
        if (sh_pop[k] < 0) continue;
        const EstOp op = sh_ops[sh_pop[k]];
        const EstIn* in = sh_in + op.in_begin;
        const int p = op.p, m = op.k - (p >= 0 ? 1 : 0), a = sh_pa[k];
        const int la = a + (p >= 0 && a >= p ? 1 : 0);
        const EstIn& x = in[la];
        const int cx = cond_digit(c, x.slot, w);
        const int32_t sv = __ldg(x.s + ro + cx);
        sh_cac[k][t % nchunk] = sv < 0 ? uint32_t(-int64_t(sv)) : uint32_t(sv);
        const int rpos = __ldg(rank_row(x, x, A.d, item.row, w) + cx);
        i128 v = i128(sv);
        bool o1 = false;
        for (int b = 0; b < m && v != 0; b++) {  // the others are leaves: G is a cached suffix sum
          if (b == a) continue;
          const EstIn& y = in[b + (p >= 0 && b >= p ? 1 : 0)];
          const int q = __ldg(rank_row(x, y, A.d, item.row, w) + rpos);
          o1 |= mul_s(v, suf[int64_t(y.suf) * W1 + q], &v);
        }
        sh_cval[k][t % nchunk] = v;
        if (o1) atomicOr(sh_flag, 1);
      }
      __syncthreads();
    }

    i128 acc = 0;
    bool ovf = false;
    // a split root: one pass, the root's sorted positions [r_lo, r_hi) of this item
    const int c_end = sb.split ? item.c0 + 1 : item.c1;
    const int r_lo = sb.split ? item.c0 : 0, r_hi = sb.split ? item.c1 : w;
    for (int c = item.c0; c < c_end; c++) {
      if (pre_ok) {
        if (sh_skip[c - item.c0]) continue;  // block-uniform
      } else {
        bool zero = false;
        for (int q = 0; q < sh_ncond; q++) zero |= __ldg(sh_cond[q] + cond_digit(c, sh_cond_k[q], w)) == 0;
        if (zero) continue;  // block-uniform
      }
      for (int o = 0; o < sb.n_ops; o++) {
        const EstOp op = sh_ops[o];
        const EstIn* in = sh_in + op.in_begin;
        const int k = op.k, p = op.p;
        const int m = k - (p >= 0 ? 1 : 0);
        // 1. suffix sums of messages arriving from non-leaf children
        for (int a = 0; a < m; a++) {
          const EstIn& x = in[a + (p >= 0 && a >= p ? 1 : 0)];
          if (x.kind == kInCache) {
            S* sl = suf + int64_t(x.suf) * W1;
            const i128* gm = A.cache + (int64_t(x.slot) * A.d + item.row) * w;
            const int32_t* perm = x.perm + ro;
            bool so1 = false;
            for (int r = tid; r < w; r += T) {
              const i128 v = gm[__ldg(perm + r)];
              so1 |= !store_fits(v, sl);
              sl[r] = S(v);
            }
            if (so1) atomicOr(sh_flag, 2);
            if (tid == 0) sl[w] = 0;
            __syncthreads();
            block_scan(sl, w, /*reverse=*/true, bs);
            continue;
          }
          if (x.kind != kInSlot) continue;
          S* sl = suf + int64_t(x.suf) * W1;
          const S* msg = slots + int64_t(x.slot) * w;
          const int32_t* perm = x.perm + ro;
          for (int r0 = tid; r0 < w; r0 += kIlp * T) {  // independent loads first, then the gathers
            int jj[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; u++) jj[u] = r0 + u * T < w ? __ldg(perm + r0 + u * T) : 0;
            S vv[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; u++) vv[u] = msg[jj[u]];
#pragma unroll
            for (int u = 0; u < kIlp; u++)
              if (r0 + u * T < w) sl[r0 + u * T] = vv[u];
          }
          if (tid == 0) sl[w] = 0;
          __syncthreads();
          block_scan(sl, w, /*reverse=*/true, bs);
        }
        // 2a. conditioned inputs: |s[c]| and their single "attains the minimum" term
        const int pk = pre_ok ? (sh_pop[0] == o ? 0 : (sh_pop[1] == o ? 1 : -1)) : -1;
        if (pk >= 0) {  // precomputed in the prologue
          if (tid == 0) {
            sh_ac[sh_pa[pk]] = sh_cac[pk][c - item.c0];
            sh_val[sh_pa[pk]] = sh_cval[pk][c - item.c0];
          }
          __syncthreads();
        } else {
          if (tid < m) {
            const EstIn& x = in[tid + (p >= 0 && tid >= p ? 1 : 0)];
            if (x.kind == kInCond) {
              const int32_t v = __ldg(x.s + ro + cond_digit(c, x.slot, w));
              sh_ac[tid] = v < 0 ? uint32_t(-int64_t(v)) : uint32_t(v);
            }
          }
          __syncthreads();
        }
        if (pk < 0 && tid < m) {
          const int la = tid + (p >= 0 && tid >= p ? 1 : 0);
          const EstIn& x = in[la];
          if (x.kind == kInCond) {
            // its cross ranks are the cached ones at its bucket's sorted position
            const int cx = cond_digit(c, x.slot, w);
            const int rpos = __ldg(rank_row(x, x, A.d, item.row, w) + cx);
            const uint32_t tau = sh_ac[tid];
            i128 v = i128(__ldg(x.s + ro + cx));
            bool o1 = false;
            for (int b = 0; b < m; b++) {
              if (b == tid) continue;
              const int lb = b + (p >= 0 && b >= p ? 1 : 0);
              const EstIn& y = in[lb];
              const bool strict = lb < la;
              if (v != 0) {
                if (y.kind == kInCond) {
                  if (!(strict ? sh_ac[b] > tau : sh_ac[b] >= tau)) v = 0;
                } else {
                  const int q = __ldg(rank_row(x, y, A.d, item.row, w) + rpos);
                  o1 |= mul_s(v, suf[int64_t(y.suf) * W1 + q], &v);
                }
              }
            }
            sh_val[tid] = v;
            if (o1) atomicOr(sh_flag, 1);
          }
        }
        __syncthreads();
        // 2b. other inputs: s_l m_l prod_{l' != l, p} G_l'(|s_l|) in l's sorted order
        i128 root_part = 0;
        for (int a = 0; a < m; a++) {
          const int la = a + (p >= 0 && a >= p ? 1 : 0);
          const EstIn& x = in[la];
          if (x.kind == kInCond) {
            if (p < 0 && tid == 0) ovf |= add_ovf(root_part, sh_val[a], &root_part);
            continue;
          }
          const int32_t* perm = x.perm + ro;
          const uint32_t* absa = x.abs + ro;
          const S* msg = x.kind == kInSlot ? slots + int64_t(x.slot) * w : nullptr;
          const i128* gm = x.kind == kInCache ? A.cache + (int64_t(x.slot) * A.d + item.row) * w : nullptr;
          S* pl = pre + int64_t(a) * W1;
          bool o2 = false, so2 = false;
          const int rb = p < 0 ? r_lo : 0, re = p < 0 ? r_hi : w;  // (a split sub-plan's op is its root)
          for (int r0 = rb + tid; r0 < re; r0 += kIlp * T) {
            int jj[kIlp];
            bool ok[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; u++) {
              ok[u] = r0 + u * T < re;
              jj[u] = ok[u] ? __ldg(perm + r0 + u * T) : 0;
            }
            int64_t sv[kIlp], mv[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; u++) {
              sv[u] = __ldg(x.s + ro + jj[u]);
              mv[u] = (msg || gm) ? int64_t(0) : int64_t(__ldg(x.msk + ro + jj[u]));
            }
            i128 v[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; u++) {
              if (msg) o2 |= mul_s(i128(sv[u]), msg[jj[u]], &v[u]);
              else if (gm) o2 |= mul_s(i128(sv[u]), gm[jj[u]], &v[u]);
              else v[u] = i128(sv[u]) * i128(mv[u]);  // |int32 * int32| < 2^62
              if (!ok[u]) v[u] = 0;
            }
            for (int b = 0; b < m; b++) {
              if (b == a) continue;
              const int lb = b + (p >= 0 && b >= p ? 1 : 0);
              const EstIn& y = in[lb];
              if (y.kind == kInCond) {
#pragma unroll
                for (int u = 0; u < kIlp; u++) {
                  const uint32_t tau = ok[u] ? __ldg(absa + r0 + u * T) : 0u;
                  if (!(lb < la ? sh_ac[b] > tau : sh_ac[b] >= tau)) v[u] = 0;
                }
              } else {
                const int32_t* rrow = rank_row(x, y, A.d, item.row, w);
                int qq[kIlp];
#pragma unroll
                for (int u = 0; u < kIlp; u++) qq[u] = ok[u] ? __ldg(rrow + r0 + u * T) : 0;
                S gg[kIlp];
#pragma unroll
                for (int u = 0; u < kIlp; u++) gg[u] = suf[int64_t(y.suf) * W1 + qq[u]];
#pragma unroll
                for (int u = 0; u < kIlp; u++)
                  if (v[u] != 0) o2 |= mul_s(v[u], gg[u], &v[u]);
              }
            }
#pragma unroll
            for (int u = 0; u < kIlp; u++) {
              if (!ok[u]) continue;
              if (p < 0) {
                o2 |= add_ovf(root_part, v[u], &root_part);
              } else {
                so2 |= !store_fits(v[u], pl);
                pl[r0 + u * T + 1] = S(v[u]);
              }
            }
          }
          if (o2) atomicOr(sh_flag, 1);
          if (so2) atomicOr(sh_flag, 2);
          if (p >= 0) {
            if (tid == 0) pl[0] = 0;
            __syncthreads();
            block_scan(pl + 1, w, /*reverse=*/false, bs);
          }
        }
        if (p < 0) {
          bool o4 = false;
          const i128 scal = block_sum(root_part, &o4, bs);
          ovf |= o4 | add_ovf(acc, scal, &acc);
          continue;
        }
        // 3. message to the parent, evaluated in the output sketch's sorted order
        {
          const EstIn& xp = in[p];
          const int32_t* permp = xp.perm + ro;
          const uint32_t* absp = xp.abs + ro;
          S* out = op.out_slot >= 0 ? slots + int64_t(op.out_slot) * w : nullptr;  // else gout
          bool o3 = false, so3 = false;
          for (int r0 = tid; r0 < w; r0 += kIlp * T) {
            int jp[kIlp];
            uint32_t tau[kIlp];
            bool ok[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; u++) {
              ok[u] = r0 + u * T < w;
              jp[u] = ok[u] ? __ldg(permp + r0 + u * T) : 0;
              tau[u] = ok[u] ? __ldg(absp + r0 + u * T) : 0u;
            }
            i128 t[kIlp], add[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; u++) {
              t[u] = i128(__ldg(xp.s + ro + jp[u]));
              add[u] = 0;
            }
            for (int a = 0; a < m; a++) {
              const int la = a + (a >= p ? 1 : 0);
              const EstIn& x = in[la];
              if (x.kind == kInCond) {
#pragma unroll
                for (int u = 0; u < kIlp; u++) {
                  if (t[u] != 0 && !(la < p ? sh_ac[a] > tau[u] : sh_ac[a] >= tau[u])) t[u] = 0;
                  if (la > p ? sh_ac[a] < tau[u] : sh_ac[a] <= tau[u]) o3 |= add_ovf(add[u], sh_val[a], &add[u]);
                }
              } else {
                const int32_t* rrow = rank_row(xp, x, A.d, item.row, w);
                int qq[kIlp];
#pragma unroll
                for (int u = 0; u < kIlp; u++) qq[u] = ok[u] ? __ldg(rrow + r0 + u * T) : 0;
                S gs[kIlp], gp[kIlp];
#pragma unroll
                for (int u = 0; u < kIlp; u++) {
                  gs[u] = suf[int64_t(x.suf) * W1 + qq[u]];
                  gp[u] = pre[int64_t(a) * W1 + qq[u]];
                }
#pragma unroll
                for (int u = 0; u < kIlp; u++) {
                  if (t[u] != 0) o3 |= mul_s(t[u], gs[u], &t[u]);
                  o3 |= add_ovf(add[u], i128(gp[u]), &add[u]);
                }
              }
            }
#pragma unroll
            for (int u = 0; u < kIlp; u++) {
              if (!ok[u]) continue;
              o3 |= add_ovf(t[u], add[u], &t[u]);
              if (out) {
                so3 |= !store_fits(t[u], out);
                out[jp[u]] = S(t[u]);
              } else {
                gout[jp[u]] = t[u];
              }
            }
          }
          if (o3) atomicOr(sh_flag, 1);
          if (so3) atomicOr(sh_flag, 2);
          __syncthreads();
        }
      }
    }
    __syncthreads();
    const int fl = sh_flag[0];
    if (tid == 0) {
      A.partial[it] = acc;
      // storage overflow: recompute with int128 storage; else arithmetic overflow is final
      A.partial_ovf[it] = (fl & 2) ? 2 : ((ovf || (fl & 1)) ? 1 : 0);
      if (gout) A.cache_ovf[int64_t(sb.job) * A.d + item.row] = (fl & 1) ? 1 : 0;
    }
    __syncthreads();
  }
}

// One CTA per sub-plan, one thread per sketch row: the row's sum over its items (conditioning
// chunks or column chunks), then thread 0 takes the exact median and rounds once.
constexpr int kFinalizeThreads = 64;  // >= CMP_MAX_D

__global__ void __launch_bounds__(kFinalizeThreads) k_estimate_finalize(const __grid_constant__ EstArgs A,
                                                                        double* __restrict__ est,
                                                                        int64_t* __restrict__ row_est,
                                                                        int64_t* __restrict__ wide_rows) {
  __shared__ i128 rows[CMP_MAX_D];
  __shared__ int32_t any_ovf, lost;
  const int64_t q = blockIdx.x;
  const EstSub sb = A.subs[q];
  const int d = A.d, i = threadIdx.x;
  if (i == 0) any_ovf = lost = 0;
  __syncthreads();
  bool ovf = false;
  if (i < d) {
    i128 s = 0;
    if (sb.single) {
      s = i128(*sb.sv);
    } else if (sb.star >= 0) {  // a star: gather T_a(S \ {a}) over its leaf edges a
      const StarFam F = A.star[sb.star];
      const int k = F.K - 1;
      for (int a = 0; a < F.K; a++) {
        if (!((sb.sbits >> a) & 1u)) continue;
        const uint32_t V = (sb.sbits & ((1u << a) - 1u)) | ((sb.sbits >> (a + 1)) << a);
        const int64_t idx = F.t_off + ((int64_t(i) * F.K + a) << k) + V;
        ovf |= A.star_tf[idx] != 0;
        ovf |= add_ovf(s, A.star_t[idx], &s);
      }
    } else {
      const int64_t it0 = int64_t(sb.item_begin) + int64_t(i) * sb.n_chunks;
      for (int ch = 0; ch < sb.n_chunks; ch++) {
        ovf |= A.partial_ovf[it0 + ch] != 0;
        ovf |= add_ovf(s, A.partial[it0 + ch], &s);
      }
    }
    rows[i] = s;
    if (row_est) {
      row_est[(q * d + i) * 2] = int64_t(uint64_t(u128(s)));
      row_est[(q * d + i) * 2 + 1] = int64_t(uint64_t(u128(s) >> 64));
    }
    if (wide_rows)  // sign-extended; rows beyond int128 are overwritten by the exact tier
      for (int l = 0; l < kWideLimbs; l++)
        wide_rows[(q * d + i) * kWideLimbs + l] = l == 0 ? int64_t(uint64_t(u128(s)))
                                                  : l == 1 ? int64_t(uint64_t(u128(s) >> 64)) : (s < 0 ? -1 : 0);
    if (ovf) atomicOr(&any_ovf, 1);
  }
  __syncthreads();
  // Exact tier: the rows beyond int128 of a sub-plan are queued and evaluated again modulo
  // the primes, one unit per conditioning chunk of the row (its units are consecutive); its
  // other rows are kept as they are for the median.
  if (A.wide && i < d && any_ovf) {
    int32_t slot = -1;
    if (ovf) {
      const uint32_t k = atomicAdd(A.wide_queue, 1u);
      const bool lat = wide_star_row(A, q);
      const uint32_t nch = uint32_t(wide_row_units(A, q));
      const uint32_t cap = uint32_t(A.wide_unit_cap);
      // no reservation once the units are used up (the counter cannot wrap)
      const bool room = k < uint32_t(A.wide_qcap) && *reinterpret_cast<volatile uint32_t*>(A.wide_queue + 2) < cap;
      const uint32_t u0 = room ? atomicAdd(A.wide_queue + 2, nch) : cap;
      if (u0 < cap && nch <= cap - u0) {
        A.wide_queue[4 + k] = uint32_t(q * d + i);
        A.wide_row_start[k] = int32_t(u0);
        for (uint32_t c = 0; c < nch; c++) A.wide_units[u0 + c] = (uint64_t(k) << 32) | (lat ? kUnitLattice : c);
        if (lat) {  // its lattice sums start from 0 (residues) and 0.0 (bound)
          for (int j = 0; j <= kWideMods; j++) A.wide_part[int64_t(u0) * (kWideMods + 1) + j] = 0;
          atomicAdd(A.wide_star_cnt + int64_t(sb.star) * d + i, 1u);
        }
        slot = int32_t(k);
      } else {
        if (k < uint32_t(A.wide_qcap)) A.wide_row_start[k] = -1;
        for (uint32_t c = u0; c < cap; c++) A.wide_units[c] = ~0ull;  // the part of the cap it took
        atomicOr(&lost, 1);
      }
    }
    A.wide_slot[q * d + i] = slot;
    A.wide_in[q * d + i] = rows[i];
  }
  __syncthreads();
  if (i != 0) return;
  if (any_ovf) {
    if (A.wide && !lost) {  // the exact tier writes est[q]
      const uint32_t k = atomicAdd(A.wide_queue + 1, 1u);
      A.wide_queue[4 + A.wide_qcap + k] = uint32_t(q);
      return;
    }
    est[q] = __longlong_as_double(0x7ff8000000000000ll);
    set_status(A.status, CMP_EOVERFLOW);
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
  est[q] = __dmul_rn(med, sb.scale);  // sampled tables: one rounded product (scale 1 is exact)
}

cudaError_t launch_estimate(const EstArgs& a, const EstPlanHdr& H, double* est, int64_t* row_est, cudaStream_t st,
                            int64_t* wide_rows) {
  // cached subtree messages, one launch per level, in int128 storage
  // three register budgets: 1024 threads (one CTA per SM), 512 (wider ILP), 256 (four CTAs
  // per SM: more items in flight when each is bound by its barriers, e.g. conditioned cycles)
  int64_t lo = 0;
  for (int l = 0; l < H.n_levels; l++) {
    const int64_t hi = H.lvl_end[l];
    if (a.threads > 512) k_estimate_items<i128, 1, 1024><<<a.grid, a.threads, 0, st>>>(a, 0, lo, hi);
    else if (a.threads > 256) k_estimate_items<i128, 2, 512><<<a.grid, a.threads, 0, st>>>(a, 0, lo, hi);
    else k_estimate_items<i128, 1, 256, 4><<<a.grid, a.threads, 0, st>>>(a, 0, lo, hi);
    lo = hi;
  }
  if (a.n_gen_items > a.n_job_items) {
    // int64 storage first; items whose stored values left int64 are recomputed in int128
    const int64_t b = a.n_job_items, e = a.n_gen_items;
    if (a.threads > 512) {
      k_estimate_items<int64_t, 2, 1024><<<a.grid, a.threads, 0, st>>>(a, 0, b, e);
      k_estimate_items<i128, 1, 1024><<<a.grid, a.threads, 0, st>>>(a, 1, b, e);
    } else if (a.threads > 256) {
      k_estimate_items<int64_t, 4, 512><<<a.grid, a.threads, 0, st>>>(a, 0, b, e);
      k_estimate_items<i128, 2, 512><<<a.grid, a.threads, 0, st>>>(a, 1, b, e);
    } else {
      k_estimate_items<int64_t, 2, 256, 4><<<a.grid, a.threads, 0, st>>>(a, 0, b, e);
      k_estimate_items<i128, 1, 256, 4><<<a.grid, a.threads, 0, st>>>(a, 1, b, e);
    }
  }
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (a.n_tri > 0) {
    const cudaError_t e = launch_estimate_tri(a, st);
    if (e != cudaSuccess) return e;
  }
  if (a.n_star_units > 0) {
    const cudaError_t e = launch_estimate_star(a, st);
    if (e != cudaSuccess) return e;
  }
  if (a.n_sub > 0) {
    if (a.wide && cudaMemsetAsync(a.wide_queue, 0, 4 * sizeof(uint32_t), st) != cudaSuccess) return cudaGetLastError();
    if (a.wide && a.n_star > 0 &&  // the star-row counters and flags (three arrays, back to back)
        cudaMemsetAsync(a.wide_star_cnt, 0,
                        size_t(reinterpret_cast<unsigned char*>(a.wide_star_kmax) -
                               reinterpret_cast<unsigned char*>(a.wide_star_cnt)) +
                            sizeof(int32_t) * size_t(a.n_star) * size_t(a.d),
                        st) != cudaSuccess)
      return cudaGetLastError();
    k_estimate_finalize<<<unsigned(a.n_sub), kFinalizeThreads, 0, st>>>(a, est, row_est, wide_rows);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_estimate_wide(a, est, wide_rows, st);
  }
  return cudaSuccess;
}

}  // namespace cmpk
