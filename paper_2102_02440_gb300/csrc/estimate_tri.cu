// Triangle sub-plans: the conditioned sum of a sub-plan whose only cycle is a triangle,
// evaluated as batched dominance sums instead of one tree contraction per conditioning
// value (the estimate itself is the contraction of the sketch-merging estimate, Sec. 4.2
// merge equation iterated over a table's joins, Sec. 3.2 per-row sums and median).
//
// Setting.  Tables U, V, W form the cycle; e* = U-V is the conditioned edge (bucket c),
// eU = U-W (bucket k) and eV = V-W (bucket i).  Every other table is a leaf joined to one
// of the three.  "x beats y" is the merge order on (|value|, edge id): smaller magnitude
// first, the lower edge id first on ties.  It is a total order, so it is transitive.
//
//  * Fix c.  U's message to W over eU is then a clamp.  At buckets k whose U-sketch value
//    on eU beats s_U*(c) it equals phiU[k], U's message with e* left out.  At the other
//    buckets it is the scalar psiU(c), U's message along e* with eU left out, read at c.
//    (The losing fixed input never attains the minimum, and a leaf value that beats the
//    winner beats the loser too.)  The first kind is a prefix of U's presorted order of its
//    eU sketch, of length rU(c).  The same holds for V.
//  * For fixed (k, i), W's merged value summed over W's leaves is f[k] (W's message along eU
//    with eV left out) when W's eU value at k beats its eV value at i, and g[i] otherwise.
//
// Let u and v be the positions of k and i in U's and V's presorted orders.  Then
//   E_row = sum_c sum_{u,v} mU_c(u) mV_c(v) Cell(u,v),   Cell(u,v) = sel(u,v) ? f_u : g_v.
// For one c, sum_u mU_c(u) Cell(u,v) = A_v(rU) + psiU(c) (Tot_v - B_v(rU)).  Here
//   A_v(r) = sum_{u<r} phiU_u Cell(u,v),   B_v(r) = sum_{u<r} Cell(u,v),   Tot_v = B_v(w).
// Conditioning values with equal rU form a group.  A group adds A_v H1_v - B_v H2_v to
// column v, and Tot_v H2_v after all rows, where
//   H1_v = sum_c mV_c(v),   H2_v = sum_c psiU(c) mV_c(v),
//   mV_c(v) = phiV_v if v < rV(c), else psiV(c).
// So H1 and H2 are prefix sums over the group's values sorted by rV.
//
// Rows between consecutive group ranks form a batch.  Sorted by W's eU key within the batch,
// the batch's share of A_v and B_v is a prefix sum read at one binary-searched position.
// The cost per sketch row is O(w G log w) for G distinct row-side ranks, against O(w^2)
// for one contraction per c.  Per sketch row, the row side is whichever of U, V has
// fewer distinct magnitudes in its conditioned sketch; G is at most that count.
//
// Leaves at a node.  With the fixed input a at value x, the node's message is
//   x * prod_l G_l(x) + sum_l PRE_l[q_l(x)].
//   - G_l(x) is the sum of leaf l's message over the buckets that x beats: a suffix of l's
//     sorted order starting at q_l(x), the number of l's values that beat x.
//   - PRE_l holds prefix sums of the "leaf l attains the minimum" terms: value times leaf
//     message times the other leaves' G at that value.
// All arithmetic is exact int128 with overflow checks; an overflow makes the row
// estimate NaN with CMP_EOVERFLOW, as on the generic path.
#include <cuda_runtime.h>

#include "est_arith.cuh"

namespace cmpk {
namespace {

__device__ __forceinline__ bool sub_ovf(i128 a, i128 b, i128* r) {
  const i128 s = i128(u128(a) - u128(b));
  *r = s;
  return ((a ^ b) & (a ^ s)) < 0;
}

__device__ __forceinline__ uint32_t mag32(int32_t v) { return v < 0 ? uint32_t(-int64_t(v)) : uint32_t(v); }

// Regions of one triangle row's scratch (see tri_layout).
struct TriPtrs {
  int32_t* hdr;  // [0] groups G, [1] queries, [2] overflow in the preparation
  i128* vec;     // [6][w]: phiU psiU phiV psiV f g, in bucket order
  i128* tmp;     // [3][w]: per node
  int64_t* sg;   // [3 * max_leaves][w+1]
  i128* pre;     // [3 * max_leaves][w+1]
  uint64_t* rkx;
  i128* rpre;  // [3][w+1]: phi*f, f, phi of the row side, exclusive prefix sums
  uint64_t* cky;
  i128* ccol;  // [2][w]: phi, g of the column side
  int32_t* qs;
  int32_t* qr;
  i128* qpre;  // [3][w+1]: psiR, psiC, psiR*psiC, exclusive prefix sums
  int32_t* gr;
  int32_t* gqb;
};

__device__ TriPtrs tri_ptrs(unsigned char* base, int w, int max_leaves) {
  const TriLayout L = tri_layout(w, max_leaves);
  TriPtrs p;
  p.hdr = reinterpret_cast<int32_t*>(base + L.hdr);
  p.vec = reinterpret_cast<i128*>(base + L.vec);
  p.tmp = reinterpret_cast<i128*>(base + L.tmp);
  p.sg = reinterpret_cast<int64_t*>(base + L.sg);
  p.pre = reinterpret_cast<i128*>(base + L.pre);
  p.rkx = reinterpret_cast<uint64_t*>(base + L.rkx);
  p.rpre = reinterpret_cast<i128*>(base + L.rpre);
  p.cky = reinterpret_cast<uint64_t*>(base + L.cky);
  p.ccol = reinterpret_cast<i128*>(base + L.ccol);
  p.qs = reinterpret_cast<int32_t*>(base + L.qs);
  p.qr = reinterpret_cast<int32_t*>(base + L.qr);
  p.qpre = reinterpret_cast<i128*>(base + L.qpre);
  p.gr = reinterpret_cast<int32_t*>(base + L.gr);
  p.gqb = reinterpret_cast<int32_t*>(base + L.gqb);
  return p;
}

// Merge sort of key[0..n2) ascending in shared memory, n2 = E * blockDim.x: thread t sorts
// keys [t E, t E + E) in registers, then log2(blockDim.x) rounds each merge pairs of sorted
// runs; a thread finds where its E outputs start on the merge path by binary search and
// merges them sequentially.  Two barriers per round (about 20 for 4096 keys).
template <int E>
__device__ void merge_sort_reg(unsigned long long* key, int n2) {
  const int t = threadIdx.x;
  unsigned long long v[E];
#pragma unroll
  for (int e = 0; e < E; e++) v[e] = key[t * E + e];
#pragma unroll
  for (int a = 1; a < E; a++)  // insertion sort of the thread's keys
#pragma unroll
    for (int b = a; b > 0; b--)
      if (v[b - 1] > v[b]) {
        const unsigned long long x = v[b - 1];
        v[b - 1] = v[b];
        v[b] = x;
      }
  for (int width = E; width < n2; width <<= 1) {
    __syncthreads();  // every read of the previous round is done
#pragma unroll
    for (int e = 0; e < E; e++) key[t * E + e] = v[e];
    __syncthreads();
    const int start = (t * E) & ~(2 * width - 1);  // first key of the pair of runs
    const unsigned long long* A = key + start;
    const unsigned long long* B = A + width;
    const int d = t * E - start;  // outputs of this pair before this thread's
    int lo = max(0, d - width), hi = min(d, width);
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (A[mid] <= B[d - mid - 1]) lo = mid + 1;
      else hi = mid;
    }
    int i = lo, j = d - lo;
#pragma unroll
    for (int e = 0; e < E; e++) {
      const bool take_a = i < width && (j >= width || A[i] <= B[j]);
      v[e] = take_a ? A[i] : B[j];
      if (take_a) i++;
      else j++;
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; e++) key[t * E + e] = v[e];
  __syncthreads();
}

// Plain shared-memory bitonic sort (every step with a barrier), for n2 < blockDim.x.
__device__ void bitonic_sort_smem(unsigned long long* key, int n2) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
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

// key[0..n2) sorted ascending (n2 a power of two); block-wide, ends with a barrier.
__device__ void sort_keys(unsigned long long* key, int n2) {
  switch (n2 / int(blockDim.x)) {
    case 1: merge_sort_reg<1>(key, n2); break;
    case 2: merge_sort_reg<2>(key, n2); break;
    case 4: merge_sort_reg<4>(key, n2); break;
    case 8: merge_sort_reg<8>(key, n2); break;
    case 16: merge_sort_reg<16>(key, n2); break;
    default: bitonic_sort_smem(key, n2); break;
  }
}

// Three in-place inclusive scans of n int128 values at once (the three arrays' loads
// overlap): the blocking of block_scan (thread-contiguous segments, then warp and block
// prefixes), exact sums, bit 0 of bs.sh_flag on overflow.  sh3: [3][33] shared scratch.
__device__ void block_scan3(i128* a0, i128* a1, i128* a2, int n, BlockScratch& bs, i128 (*sh3)[33]) {
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  const int per = (n + T - 1) / T;
  const int b = min(n, tid * per), e = min(n, b + per);
  i128 s[3] = {0, 0, 0};
  bool o = false;
  for (int q = b; q < e; q++) {
    const i128 x0 = a0[q], x1 = a1[q], x2 = a2[q];
    o |= add_ovf(s[0], x0, &s[0]);
    o |= add_ovf(s[1], x1, &s[1]);
    o |= add_ovf(s[2], x2, &s[2]);
  }
  i128 incl[3] = {s[0], s[1], s[2]};
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
    for (int m = 0; m < 3; m++) {
      const int64_t lo = __shfl_up_sync(0xffffffffu, int64_t(incl[m]), off);
      const int64_t hi = __shfl_up_sync(0xffffffffu, int64_t(incl[m] >> 64), off);
      const i128 other = (i128(hi) << 64) | i128(uint64_t(lo));
      i128 r;
      const bool ob = add_ovf(incl[m], other, &r);
      if (lane >= off) {
        o |= ob;
        incl[m] = r;
      }
    }
  }
  if (lane == 31)
    for (int m = 0; m < 3; m++) sh3[m][warp] = incl[m];
  __syncthreads();
  if (tid < 3) {
    i128 t = 0;
    bool oo = false;
    for (int i = 0; i < nw; i++) {
      const i128 v = sh3[tid][i];
      sh3[tid][i] = t;
      oo |= add_ovf(t, v, &t);
    }
    if (oo) atomicOr(bs.sh_flag, 1);
  }
  __syncthreads();
  i128 run[3];
#pragma unroll
  for (int m = 0; m < 3; m++) o |= add_ovf(sh3[m][warp], incl[m] - s[m], &run[m]);  // incl - s: a partial sum
  for (int q = b; q < e; q++) {
    const i128 x0 = a0[q], x1 = a1[q], x2 = a2[q];
    o |= add_ovf(run[0], x0, &run[0]);
    o |= add_ovf(run[1], x1, &run[1]);
    o |= add_ovf(run[2], x2, &run[2]);
    a0[q] = run[0];
    a1[q] = run[1];
    a2[q] = run[2];
  }
  if (o) atomicOr(bs.sh_flag, 1);
  __syncthreads();
}

// Copies a presorted magnitude row into shared memory (block-wide, ends with a barrier).
__device__ void stage_row(const uint32_t* __restrict__ src, uint32_t* dst, int w) {
  for (int r = threadIdx.x; r < w; r += blockDim.x) dst[r] = __ldg(src + r);
  __syncthreads();
}

// First position q in the sorted shared-memory row a[0..w) with a[q] > tau (strict) or
// a[q] >= tau: the number of the row's values that beat tau.
__device__ __forceinline__ int rank_sh(const uint32_t* a, int w, uint32_t tau, bool strict) {
  int lo = 0, hi = w;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const uint32_t v = a[mid];
    if (strict ? v <= tau : v < tau) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Message of triangle node n with the fixed input a (every input but ia, ib is a leaf),
// for every bucket of a's edge: out[j] = x prod_l SG_l[q_l] + sum_l PRE_l[q_l], one leaf
// at a time with the leaf's magnitudes staged in shared memory (stage: w uint32).
__device__ void node_msg(const EstArgs& A, const TriNode& nd, int n, int a, const TriPtrs& P, int64_t ro,
                         i128* __restrict__ out, i128* __restrict__ tmp, uint32_t* stage, int32_t* flag) {
  const int w = A.w, T = blockDim.x;
  const int64_t W1 = int64_t(w) + 1;
  const EstIn* in = A.inputs + nd.in_begin;
  const int32_t* __restrict__ sa = in[a].s + ro;
  bool o = false;
  for (int j = threadIdx.x; j < w; j += T) {
    out[j] = i128(__ldg(sa + j));
    tmp[j] = 0;
  }
  constexpr int U = 2;  // buckets per thread in flight: their loads are issued together
  for (int l = 0, li = 0; l < nd.k; l++) {
    if (l == nd.ia || l == nd.ib) continue;
    __syncthreads();  // the previous leaf's readers are done with the stage
    stage_row(in[l].abs + ro, stage, w);
    const int64_t slot = (int64_t(n) * A.tri_max_leaves + li) * W1;
    const int64_t* __restrict__ sg = P.sg + slot;
    const i128* __restrict__ pre = P.pre + slot;
    const bool before = l < a;
    for (int j0 = threadIdx.x; j0 < w; j0 += U * T) {
      int q[U];
      i128 v[U], acc[U], g[U], p[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int j = j0 + u * T;
        // leaf values that beat x: |y| < |x|, or |y| == |x| with l before a
        q[u] = j < w ? rank_sh(stage, w, mag32(__ldg(sa + j)), before) : 0;
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int j = j0 + u * T;
        v[u] = j < w ? out[j] : 0;
        acc[u] = j < w ? tmp[j] : 0;
        g[u] = sg[q[u]];
        p[u] = pre[q[u]];
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int j = j0 + u * T;
        if (j >= w) continue;
        i128 x = v[u], y = acc[u];
        if (x != 0) o |= mul_ovf_64(x, int64_t(g[u]), &x);
        o |= add_ovf(y, p[u], &y);
        out[j] = x;
        tmp[j] = y;
      }
    }
    li++;
  }
  for (int j = threadIdx.x; j < w; j += T) {
    i128 v = out[j];
    o |= add_ovf(v, tmp[j], &v);
    out[j] = v;
  }
  if (o) atomicOr(flag, 1);
  __syncthreads();
}

// Exclusive scan of the 0/1 flags at[0..n) (thread-contiguous ranges).  Returns this
// thread's first output index and writes the total to *total.
__device__ int block_count_base(const int32_t* at, int n, int32_t* sh_w, int32_t* total) {
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  const int per = (n + T - 1) / T;
  const int b = min(n, tid * per), e = min(n, b + per);
  int cnt = 0;
  for (int q = b; q < e; q++) cnt += at[q] != 0;
  int incl = cnt;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += o;
  }
  if (lane == 31) sh_w[warp] = incl;
  __syncthreads();
  if (tid == 0) {
    int t = 0;
    for (int i = 0; i < nw; i++) {
      const int v = sh_w[i];
      sh_w[i] = t;
      t += v;
    }
    *total = t;
  }
  __syncthreads();
  const int base = sh_w[warp] + incl - cnt;
  __syncthreads();
  return base;
}

}  // namespace

// One CTA per (triangle row of the wave starting at tr0, node n of the triangle): node n's
// leaf suffix sums, its leaves' "attains the minimum" prefix sums and its two messages.
// The three nodes of a row are independent, so they run on three SMs; the node's overflow
// flag goes to hdr[3 + n] (k_tri_prep folds it into the row's flag).
__global__ void __launch_bounds__(1024) k_tri_nodes(const __grid_constant__ EstArgs A, int64_t tr0) {
  extern __shared__ uint32_t stage[];  // [w]: one staged magnitude row
  __shared__ i128 sh_i128[33];
  __shared__ int32_t sh_flag[1];
  BlockScratch bs{sh_i128, sh_flag};
  const int w = A.w, d = A.d, tid = threadIdx.x, T = blockDim.x;
  const int64_t W1 = int64_t(w) + 1;
  const int64_t slot = blockIdx.x / 3;
  const int n = int(blockIdx.x % 3);
  const int64_t tr = tr0 + slot;
  const TriSub ts = A.tri[tr / d];
  const TriNode nd = ts.node[n];
  const int64_t ro = (tr % d) * int64_t(w);
  const TriPtrs P = tri_ptrs(A.tri_scratch + slot * A.tri_row_bytes, w, A.tri_max_leaves);
  i128* tmp = P.tmp + int64_t(n) * w;
  const EstIn* inputs = A.inputs;
  if (tid == 0) sh_flag[0] = 0;
  __syncthreads();

  // ---- leaves: suffix sums of each leaf's message in its sketch's sorted order
  {
    for (int l = 0, li = 0; l < nd.k; l++) {
      if (l == nd.ia || l == nd.ib) continue;
      const EstIn& x = inputs[nd.in_begin + l];
      int64_t* sg = P.sg + (int64_t(n) * A.tri_max_leaves + li) * W1;
      const int32_t* perm = x.perm + ro;
      for (int r = tid; r < w; r += T) sg[r] = __ldg(x.msk + ro + __ldg(perm + r));
      if (tid == 0) sg[w] = 0;
      __syncthreads();
      block_scan(sg, w, /*reverse=*/true, bs);
      li++;
    }
  }
  // ---- leaves: prefix sums of the terms in which leaf l attains the minimum: value times
  // leaf message, times every other leaf's suffix sum at that value (other leaf staged)
  {
    for (int l = 0, li = 0; l < nd.k; l++) {
      if (l == nd.ia || l == nd.ib) continue;
      const EstIn& x = inputs[nd.in_begin + l];
      i128* pre = P.pre + (int64_t(n) * A.tri_max_leaves + li) * W1;
      const int32_t* perm = x.perm + ro;
      for (int r = tid; r < w; r += T) {
        const int j = __ldg(perm + r);
        pre[r + 1] = i128(int64_t(__ldg(x.s + ro + j)) * int64_t(__ldg(x.msk + ro + j)));  // |int32 * int32| < 2^62
      }
      bool o = false;
      for (int l2 = 0, li2 = 0; l2 < nd.k; l2++) {
        if (l2 == nd.ia || l2 == nd.ib) continue;
        if (l2 != l) {
          __syncthreads();
          stage_row(inputs[nd.in_begin + l2].abs + ro, stage, w);
          const int64_t* sg2 = P.sg + (int64_t(n) * A.tri_max_leaves + li2) * W1;
          for (int r = tid; r < w; r += T) {
            i128 v = pre[r + 1];
            if (v == 0) continue;
            const uint32_t tau = mag32(__ldg(x.s + ro + __ldg(perm + r)));
            o |= mul_ovf_64(v, sg2[rank_sh(stage, w, tau, l2 < l)], &v);
            pre[r + 1] = v;
          }
        }
        li2++;
      }
      if (o) atomicOr(sh_flag, 1);
      if (tid == 0) pre[0] = 0;
      __syncthreads();
      block_scan(pre + 1, w, /*reverse=*/false, bs);
      li++;
    }
  }
  // ---- the node's two messages, in bucket order
  node_msg(A, nd, n, nd.ia, P, ro, P.vec + int64_t(2 * n) * w, tmp, stage, sh_flag);
  node_msg(A, nd, n, nd.ib, P, ro, P.vec + int64_t(2 * n + 1) * w, tmp, stage, sh_flag);
  if (tid == 0) P.hdr[3 + n] = sh_flag[0] != 0;
}

// One CTA per triangle row (sub-plan, sketch row) of the wave starting at tr0.
// sep: the dynamic shared memory also holds two staged rows after the group ranks.
__global__ void __launch_bounds__(1024) k_tri_prep(const __grid_constant__ EstArgs A, int64_t tr0, int sep) {
  extern __shared__ unsigned long long key[];
  __shared__ i128 sh_i128[33];
  __shared__ i128 sh_scan3[3][33];
  __shared__ int32_t sh_flag[1];
  __shared__ int32_t sh_cnt[4];
  __shared__ int32_t sh_w[32];
  BlockScratch bs{sh_i128, sh_flag};
  const int w = A.w, d = A.d, tid = threadIdx.x, T = blockDim.x;
  if (w > kTriMaxW || T != 1024) {  // the planner never sends these; sorts and group starts assume them
    if (tid == 0) set_status(A.status, CMP_EINVAL);
    return;
  }
  const int64_t W1 = int64_t(w) + 1;
  const int64_t tr = tr0 + blockIdx.x;
  const TriSub ts = A.tri[tr / d];
  const int64_t ro = (tr % d) * int64_t(w);
  const TriPtrs P = tri_ptrs(A.tri_scratch + int64_t(blockIdx.x) * A.tri_row_bytes, w, A.tri_max_leaves);
  const EstIn* inputs = A.inputs;
  int wp2 = 1;
  while (wp2 < w) wp2 <<= 1;
  if (tid == 0) {
    sh_flag[0] = 0;
    sh_cnt[0] = sh_cnt[1] = sh_cnt[2] = sh_cnt[3] = 0;
  }
  __syncthreads();

  // the node kernel's overflow flags
  if (tid == 0 && (P.hdr[3] | P.hdr[4] | P.hdr[5])) sh_flag[0] = 1;
  uint32_t* stage = reinterpret_cast<uint32_t*>(key);  // 2 * wp2 uint32 before the sorts use it
  __syncthreads();
  // ---- row side: U or V, whichever conditioned sketch has fewer distinct magnitudes
  for (int n = 0; n < 2; n++) {
    const uint32_t* ab = inputs[ts.node[n].in_begin + ts.node[n].ib].abs + ro;
    int cnt = 0;
    for (int r = tid + 1; r < w; r += T) cnt += __ldg(ab + r) != __ldg(ab + r - 1);
    if (cnt) atomicAdd(&sh_cnt[n], cnt);
  }
  __syncthreads();  // also orders the node messages before their reads below
  const bool swap = sh_cnt[1] < sh_cnt[0];
  const TriNode NR = ts.node[swap ? 1 : 0], NC = ts.node[swap ? 0 : 1], NW = ts.node[2];
  const int wR = swap ? NW.ib : NW.ia, wC = swap ? NW.ia : NW.ib;  // W's edges to R and C
  const i128* phiR = P.vec + int64_t(swap ? 2 : 0) * w;
  const i128* psiR = P.vec + int64_t(swap ? 3 : 1) * w;
  const i128* phiC = P.vec + int64_t(swap ? 0 : 2) * w;
  const i128* psiC = P.vec + int64_t(swap ? 1 : 3) * w;
  const i128* fR = P.vec + int64_t(swap ? 5 : 4) * w;
  const i128* gC = P.vec + int64_t(swap ? 4 : 5) * w;
  const bool tieR = NR.ia < NR.ib, tieC = NC.ia < NC.ib, tieW = wR < wC;
  const EstIn& Rpar = inputs[NR.in_begin + NR.ia];
  const EstIn& Rcond = inputs[NR.in_begin + NR.ib];
  const EstIn& Cpar = inputs[NC.in_begin + NC.ia];
  const EstIn& Ccond = inputs[NC.in_begin + NC.ib];
  const EstIn& Wr = inputs[NW.in_begin + wR];
  const EstIn& Wc = inputs[NW.in_begin + wC];

  // ---- queries: conditioning values with both conditioned sketch values nonzero (a zero
  // makes every merged entry at c through that table 0), sorted by (rR, rC, c).  The
  // clamp ranks (number of parent-sketch values that beat the conditioned value) are
  // searched in the staged parent rows, kept per c in qr / qs, then packed into keys.
  if (sep) {  // the staged rows have their own region: the keys are written directly
    uint32_t* stR = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(key + wp2) +
                                                align16(sizeof(int32_t) * size_t(w + 1)));
    uint32_t* stC = stR + wp2;
    for (int r = tid; r < w; r += T) {
      stR[r] = __ldg(Rpar.abs + ro + r);
      stC[r] = __ldg(Cpar.abs + ro + r);
    }
    __syncthreads();
    int cnt = 0;
    for (int c = tid; c < wp2; c += T) {
      unsigned long long kk = ~0ull;
      if (c < w) {
        const int32_t sr = __ldg(Rcond.s + ro + c), sc = __ldg(Ccond.s + ro + c);
        if (sr != 0 && sc != 0) {
          const unsigned long long qr = unsigned(rank_sh(stR, w, mag32(sr), tieR));
          const unsigned long long qs = unsigned(rank_sh(stC, w, mag32(sc), tieC));
          kk = (qr << 42) | (qs << 21) | static_cast<unsigned long long>(c);
          cnt++;
        }
      }
      key[c] = kk;
    }
    if (cnt) atomicAdd(&sh_cnt[2], cnt);
  } else {
    uint32_t* stR = stage;
    uint32_t* stC = stage + wp2;
    for (int r = tid; r < w; r += T) {
      stR[r] = __ldg(Rpar.abs + ro + r);
      stC[r] = __ldg(Cpar.abs + ro + r);
    }
    __syncthreads();
    int cnt = 0;
    for (int c = tid; c < w; c += T) {
      const int32_t sr = __ldg(Rcond.s + ro + c), sc = __ldg(Ccond.s + ro + c);
      const bool live = sr != 0 && sc != 0;
      P.qr[c] = live ? rank_sh(stR, w, mag32(sr), tieR) : -1;
      P.qs[c] = live ? rank_sh(stC, w, mag32(sc), tieC) : -1;
      cnt += live;
    }
    if (cnt) atomicAdd(&sh_cnt[2], cnt);
    __syncthreads();  // stage no longer read: the keys overwrite it
    for (int c = tid; c < wp2; c += T) {
      unsigned long long kk = ~0ull;
      if (c < w && P.qr[c] >= 0)
        kk = (static_cast<unsigned long long>(P.qr[c]) << 42) | (static_cast<unsigned long long>(P.qs[c]) << 21) |
             static_cast<unsigned long long>(c);
      key[c] = kk;
    }
  }
  __syncthreads();
  sort_keys(key, wp2);
  const int nq = sh_cnt[2];
  {
    bool o = false;
    for (int q = tid; q < nq; q += T) {
      const unsigned long long kk = key[q];
      const int c = int(kk & 0x1FFFFFull);
      P.qs[q] = int((kk >> 21) & 0x1FFFFFull);
      P.qr[q] = int(kk >> 42);
      const i128 pr = psiR[c], pc = psiC[c];
      i128 prc;
      o |= mul_ovf(pr, pc, &prc);
      P.qpre[q + 1] = pr;
      P.qpre[W1 + q + 1] = pc;
      P.qpre[2 * W1 + q + 1] = prc;
    }
    if (o) atomicOr(sh_flag, 1);
    if (tid == 0) P.qpre[0] = P.qpre[W1] = P.qpre[2 * W1] = 0;
  }
  __syncthreads();
  block_scan3(P.qpre + 1, P.qpre + W1 + 1, P.qpre + 2 * W1 + 1, nq, bs, sh_scan3);
  // groups: first query of each distinct row-side rank (flags staged in gqb)
  for (int q = tid; q < nq; q += T) P.gqb[q] = (q == 0 || P.qr[q] != P.qr[q - 1]) ? 1 : 0;
  __syncthreads();
  {
    // launched with 1024 threads: at most kTriMaxW / 1024 queries per thread
    const int per = (nq + T - 1) / T;
    const int b = min(nq, tid * per), e = min(nq, b + per);
    int starts[kTriMaxW / 1024];
    int ns = 0;
    for (int q = b; q < e; q++)
      if (P.gqb[q]) starts[ns++] = q;
    const int base = block_count_base(P.gqb, nq, sh_w, &sh_cnt[3]);  // every flag read before it returns
    for (int i = 0; i < ns; i++) {
      P.gr[base + i] = P.qr[starts[i]];
      P.gqb[base + i] = starts[i];
    }
  }
  __syncthreads();
  const int G = sh_cnt[3];
  if (tid == 0) P.gqb[G] = nq;

  // ---- rows of the row side: batch (number of group ranks <= u), then W's key, then u
  int32_t* sgr = reinterpret_cast<int32_t*>(key + wp2);  // G <= w group ranks
  for (int g = tid; g < G; g += T) sgr[g] = P.gr[g];
  __syncthreads();
  for (int u = tid; u < wp2; u += T) {
    unsigned long long kk = ~0ull;
    if (u < w) {
      const int k = __ldg(Rpar.perm + ro + u);
      const uint64_t kx = 2ull * mag32(__ldg(Wr.s + ro + k)) + (tieW ? 0ull : 1ull);
      int lo = 0, hi = G;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sgr[mid] <= u) lo = mid + 1;
        else hi = mid;
      }
      kk = (static_cast<unsigned long long>(lo) << 48) | (kx << 14) | static_cast<unsigned long long>(u);
    }
    key[u] = kk;
  }
  __syncthreads();
  sort_keys(key, wp2);
  {
    bool o = false;
    for (int q = tid; q < w; q += T) {
      const unsigned long long kk = key[q];
      const int u = int(kk & 0x3FFFull);
      const int k = __ldg(Rpar.perm + ro + u);
      P.rkx[q] = (kk >> 14) & ((1ull << 33) - 1);
      const i128 phi = phiR[k], f = fR[k];
      i128 pf;
      o |= mul_ovf(phi, f, &pf);
      P.rpre[q + 1] = pf;
      P.rpre[W1 + q + 1] = f;
      P.rpre[2 * W1 + q + 1] = phi;
    }
    if (o) atomicOr(sh_flag, 1);
    if (tid == 0) P.rpre[0] = P.rpre[W1] = P.rpre[2 * W1] = 0;
  }
  __syncthreads();
  block_scan3(P.rpre + 1, P.rpre + W1 + 1, P.rpre + 2 * W1 + 1, w, bs, sh_scan3);
  // ---- columns of the column side, in its presorted order
  for (int v = tid; v < w; v += T) {
    const int i = __ldg(Cpar.perm + ro + v);
    P.cky[v] = 2ull * mag32(__ldg(Wc.s + ro + i)) + (tieW ? 1ull : 0ull);
    P.ccol[v] = phiC[i];
    P.ccol[w + v] = gC[i];
  }
  __syncthreads();
  if (tid == 0) {
    P.hdr[0] = G;
    P.hdr[1] = nq;
    P.hdr[2] = sh_flag[0] != 0;
  }
}

// Shared memory of the staged sweep: row keys [w] u64, group ranks and group starts [w + 1]
// each (the queries' column ranks stay in global memory).
__host__ __device__ inline int64_t tri_sweep_smem(int32_t w) { return 8 * int64_t(w) + 4 * (2 * int64_t(w) + 2); }
constexpr int64_t kTriSweepSmemMax = 72 * 1024;  // staged when three CTAs per SM still fit

// One thread per column; kTriCols columns per CTA, tri_nch CTAs per triangle row.  STAGED:
// the arrays the binary searches read are first copied to shared memory.
template <bool STAGED>
__global__ void __launch_bounds__(kTriCols, 3) k_tri_sweep(const __grid_constant__ EstArgs A, int64_t tr0) {
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  __shared__ i128 sh_i128[33];
  __shared__ int32_t sh_flag[1];
  BlockScratch bs{sh_i128, sh_flag};
  const int w = A.w, tid = threadIdx.x;
  const int64_t W1 = int64_t(w) + 1;
  const int64_t slot = blockIdx.x / A.tri_nch;
  const int ch = int(blockIdx.x % A.tri_nch);
  const int64_t it = A.n_gen_items + (tr0 + slot) * A.tri_nch + ch;
  TriPtrs P = tri_ptrs(A.tri_scratch + slot * A.tri_row_bytes, w, A.tri_max_leaves);
  if (tid == 0) sh_flag[0] = 0;
  const int G = P.hdr[0];
  const int prep_ovf = P.hdr[2];
  if (STAGED) {
    uint64_t* s_rkx = reinterpret_cast<uint64_t*>(sweep_smem);
    int32_t* s_gr = reinterpret_cast<int32_t*>(s_rkx + w);
    int32_t* s_gqb = s_gr + (w + 1);
    for (int r = tid; r < w; r += kTriCols) s_rkx[r] = P.rkx[r];
    for (int g = tid; g <= G; g += kTriCols) {
      if (g < G) s_gr[g] = P.gr[g];
      s_gqb[g] = P.gqb[g];
    }
    P.rkx = s_rkx;
    P.gr = s_gr;
    P.gqb = s_gqb;
  }
  __syncthreads();
  const int v = ch * kTriCols + tid;
  i128 E = 0;
  bool o = false;
  if (v < w) {
    const uint64_t ky = P.cky[v];
    const i128 phi = P.ccol[v], g = P.ccol[w + v];
    const i128* prePF = P.rpre;
    const i128* preF = P.rpre + W1;
    const i128* prePhi = P.rpre + 2 * W1;
    const i128* qR = P.qpre;
    const i128* qC = P.qpre + W1;
    const i128* qRC = P.qpre + 2 * W1;
    i128 SA = 0, SB = 0, SC = 0, H2t = 0, t1, t2;
    int SD = 0, lo = 0;
    for (int b = 0; b <= G; b++) {
      const int hi = b < G ? P.gr[b] : w;
      // rows of the batch whose W key is below the column's: Cell = f_u there
      int a0 = lo, a1 = hi;
      while (a0 < a1) {
        const int mid = (a0 + a1) >> 1;
        if (P.rkx[mid] < ky) a0 = mid + 1;
        else a1 = mid;
      }
      if (a0 > lo) {
        o |= sub_ovf(prePF[a0], prePF[lo], &t1);
        o |= add_ovf(SA, t1, &SA);
        o |= sub_ovf(preF[a0], preF[lo], &t1);
        o |= add_ovf(SB, t1, &SB);
        o |= sub_ovf(prePhi[a0], prePhi[lo], &t1);
        o |= add_ovf(SC, t1, &SC);
        SD += a0 - lo;
      }
      if (b < G) {
        // group b: its conditioning values have row-side rank r = hi
        const int qb = P.gqb[b], qe = P.gqb[b + 1];
        int c0 = qb, c1 = qe;  // first value whose column-side rank exceeds v
        while (c0 < c1) {
          const int mid = (c0 + c1) >> 1;
          if (P.qs[mid] <= v) c0 = mid + 1;
          else c1 = mid;
        }
        i128 Av, Bv, H1, H2;
        // A = SA + g (sum_{u<r} phi_u - SC),  B = SB + g (r - SD)
        o |= sub_ovf(prePhi[hi], SC, &t1);
        o |= mul_ovf(g, t1, &t1);
        o |= add_ovf(SA, t1, &Av);
        o |= mul_ovf_64(g, int64_t(hi - SD), &t1);
        o |= add_ovf(SB, t1, &Bv);
        // H1 = phi * #{rC > v} + sum_{rC <= v} psiC,  H2 = phi * sum_{rC > v} psiR + sum_{rC <= v} psiR psiC
        o |= mul_ovf_64(phi, int64_t(qe - c0), &H1);
        o |= sub_ovf(qC[c0], qC[qb], &t1);
        o |= add_ovf(H1, t1, &H1);
        o |= sub_ovf(qR[qe], qR[c0], &t1);
        o |= mul_ovf(phi, t1, &H2);
        o |= sub_ovf(qRC[c0], qRC[qb], &t1);
        o |= add_ovf(H2, t1, &H2);
        o |= mul_ovf(Av, H1, &t1);
        o |= mul_ovf(Bv, H2, &t2);
        o |= sub_ovf(t1, t2, &t1);
        o |= add_ovf(E, t1, &E);
        o |= add_ovf(H2t, H2, &H2t);
      }
      lo = hi;
    }
    // Tot = SB + g (w - SD) after every row
    o |= mul_ovf_64(g, int64_t(w - SD), &t1);
    o |= add_ovf(SB, t1, &t1);
    o |= mul_ovf(t1, H2t, &t1);
    o |= add_ovf(E, t1, &E);
  }
  if (o) atomicOr(sh_flag, 1);
  __syncthreads();
  bool o2 = false;
  const i128 sum = block_sum(E, &o2, bs);
  if (tid == 0) {
    A.partial[it] = sum;
    A.partial_ovf[it] = (o2 || prep_ovf) ? 1 : 0;
  }
}

cudaError_t launch_estimate_tri(const EstArgs& a, cudaStream_t st) {
  if (a.n_tri <= 0 || a.tri_slots <= 0) return cudaSuccess;
  const int64_t rows = a.n_tri * a.d;
  int wp2 = 1;
  while (wp2 < a.w) wp2 <<= 1;
  // sort keys (also two staged magnitude rows before the sorts), then the group ranks, and
  // two staged rows of their own when that fits
  const int smem0 = int(sizeof(unsigned long long)) * wp2 + int(align16(sizeof(int32_t) * size_t(a.w + 1)));
  const int sep = size_t(smem0) + 2 * sizeof(uint32_t) * size_t(wp2) <= smem_optin_bytes() - 4096 ? 1 : 0;
  const int smem = smem0 + (sep ? int(2 * sizeof(uint32_t)) * wp2 : 0);
  cudaError_t e = cudaFuncSetAttribute(k_tri_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (int64_t(4) * a.w > 48 * 1024) {
    e = cudaFuncSetAttribute(k_tri_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * a.w);
    if (e != cudaSuccess) return e;
  }
  const bool staged = tri_sweep_smem(a.w) <= kTriSweepSmemMax;
  if (staged) {
    e = cudaFuncSetAttribute(k_tri_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(tri_sweep_smem(a.w)));
    if (e != cudaSuccess) return e;
  }
  for (int64_t r0 = 0; r0 < rows; r0 += a.tri_slots) {
    const int64_t n = rows - r0 < a.tri_slots ? rows - r0 : a.tri_slots;
    k_tri_nodes<<<unsigned(3 * n), 1024, size_t(4) * size_t(a.w), st>>>(a, r0);
    k_tri_prep<<<unsigned(n), 1024, smem, st>>>(a, r0, sep);
    if (staged)
      k_tri_sweep<true><<<unsigned(n * a.tri_nch), kTriCols, size_t(tri_sweep_smem(a.w)), st>>>(a, r0);
    else
      k_tri_sweep<false><<<unsigned(n * a.tri_nch), kTriCols, 0, st>>>(a, r0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cmpk
