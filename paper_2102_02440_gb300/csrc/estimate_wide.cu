// Exact tier beyond int128 of the sketch-merging estimate (Sec. 4.2 merge equation, Sec. 3.2
// median): rows whose value, or an intermediate of their evaluation, left int128 are
// evaluated again on the generic path with modular arithmetic.
//
// The contraction of a row is a polynomial in the counters: sums of products, with the
// min-abs selections of the merge decided by comparisons of presorted magnitudes only.  So
// its value E is determined exactly by E mod p_j for primes p_j whose product P exceeds 2|E|,
// and the same evaluation with absolute values in double, rounded upwards at every step, is
// an upper bound on |E|.  E is the sum of its conditioning values' terms (one term for a
// tree), so a row is split into units, one per conditioning chunk: a CTA evaluates one
// (unit, modulus) pair; the finalize sums the units' residues and bounds, rebuilds E by
// Garner's algorithm when the bound is below 2^kWideBits (< P / 2), takes the exact median
// over the d rows and rounds it once to double.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "est_arith.cuh"

namespace cmpk {

namespace {

// ---------------------------------------------------------------- arithmetic policies
// Residues modulo p = 2^62 - c (c < 2^10): a b = H 2^62 + L = L + c H (mod p), twice, then
// one conditional subtraction (the second sum is below 2^62 + 2^21 < 2p).
struct ModArith {
  uint64_t p, c;
  using V = uint64_t;
  __device__ __forceinline__ V zero() const { return 0; }
  __device__ __forceinline__ V one() const { return 1; }
  __device__ __forceinline__ V reduce63(uint64_t u) const {  // u < 2^63
    uint64_t r = (u & ((1ull << 62) - 1)) + (u >> 62) * c;
    return r >= p ? r - p : r;
  }
  __device__ __forceinline__ V from(int64_t v) const {
    if (v >= 0) return reduce63(uint64_t(v));
    const V m = reduce63(uint64_t(0) - uint64_t(v));  // |v| <= 2^63: below 2^63 + 1, reduce63 holds
    return m ? p - m : 0;
  }
  __device__ __forceinline__ V from_wide(int64_t v) const { return from(v); }
  __device__ __forceinline__ V add(V a, V b) const {
    const uint64_t s = a + b;
    return s >= p ? s - p : s;
  }
  __device__ __forceinline__ V reduce128(u128 x) const {  // any x < 2^128 (e.g. 16 products)
    const u128 H = x >> 62;                                              // < 2^66
    const u128 y = H * c + (uint64_t(x) & ((1ull << 62) - 1));           // < 2^76 + 2^62
    const uint64_t z = (uint64_t(y) & ((1ull << 62) - 1)) + uint64_t(y >> 62) * c;  // < 2^62 + 2^24
    return z >= p ? z - p : z;
  }
  __device__ __forceinline__ V mul(V a, V b) const {
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    const uint64_t L = lo & ((1ull << 62) - 1), H = (hi << 2) | (lo >> 62);  // < 2^62 each
    const u128 y = u128(H) * c + L;                                          // < 2^72 + 2^62
    const uint64_t z = (uint64_t(y) & ((1ull << 62) - 1)) + uint64_t(y >> 62) * c;
    return z >= p ? z - p : z;
  }
};

// Upper bounds of magnitudes: |sum| <= sum of |terms|, |product| = product of |factors|,
// each rounded towards +infinity.
struct BoundArith {
  using V = double;
  __device__ __forceinline__ V zero() const { return 0.0; }
  __device__ __forceinline__ V one() const { return 1.0; }
  __device__ __forceinline__ V from(int64_t v) const { return fabs(double(v)); }  // |v| < 2^53: exact
  __device__ __forceinline__ V from_wide(int64_t v) const {                      // any int64: rounded up
    return __ull2double_ru(v < 0 ? uint64_t(0) - uint64_t(v) : uint64_t(v));
  }
  __device__ __forceinline__ V add(V a, V b) const { return __dadd_ru(a, b); }
  __device__ __forceinline__ V mul(V a, V b) const { return __dmul_ru(a, b); }
};

template <class M>
__device__ __forceinline__ typename M::V shfl_up_v(typename M::V v, int off) {
  return __shfl_up_sync(0xffffffffu, v, off);
}

// Block-wide sum (result broadcast) and in-place scans of V values.
template <class M>
__device__ typename M::V block_sum_v(const M& ar, typename M::V v, typename M::V* sh) {
  using V = typename M::V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const V o = __shfl_down_sync(0xffffffffu, v, off);
    if (lane + off < 32) v = ar.add(v, o);
  }
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    V t = ar.zero();
    for (int i = 0; i < nw; i++) t = ar.add(t, sh[i]);
    sh[32] = t;
  }
  __syncthreads();
  const V r = sh[32];
  __syncthreads();
  return r;
}

template <class M>
__device__ void block_scan_v(const M& ar, typename M::V* a, int n, bool reverse, typename M::V* sh) {
  using V = typename M::V;
  const int T = blockDim.x, tid = threadIdx.x;
  const int per = (n + T - 1) / T;
  const int b = tid * per, e = min(n, b + per);
  V s = ar.zero();
  for (int q = b; q < e; q++) s = ar.add(s, a[reverse ? n - 1 - q : q]);
  const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  V incl = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const V o = shfl_up_v<M>(incl, off);
    if (lane >= off) incl = ar.add(incl, o);
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (tid == 0) {
    V t = ar.zero();
    for (int i = 0; i < nw; i++) {
      const V v = sh[i];
      sh[i] = t;
      t = ar.add(t, v);
    }
  }
  __syncthreads();
  // exclusive prefix of this thread: the warp's base plus the lanes before it
  V run = sh[warp];
  {
    const V before = shfl_up_v<M>(incl, 1);
    if (lane > 0) run = ar.add(run, before);
  }
  for (int q = b; q < e; q++) {
    const int idx = reverse ? n - 1 - q : q;
    run = ar.add(run, a[idx]);
    a[idx] = run;
  }
  __syncthreads();
}

__device__ __forceinline__ const int32_t* wrank_row(const EstIn& x, const EstIn& y, int d, int row, int w) {
  return x.rk + (int64_t(y.tslot) * d + row) * w;
}

constexpr int kWideThreads = 128;  // latency-bound contractions: more small CTAs in flight

// Conditioning chunk ch of one row of sub-plan sb (its item it0 + ch) in arithmetic ar.
template <class M>
__device__ typename M::V wide_row(const M& ar, const EstArgs& A, const EstSub& sb, int row, int ch, EstOp* sh_ops,
                                  EstIn* sh_in, typename M::V* sh, typename M::V* sh_val, uint32_t* sh_ac,
                                  unsigned char* cta) {
  using V = typename M::V;
  const int w = A.w, tid = threadIdx.x, T = blockDim.x;
  const int64_t W1 = int64_t(w) + 1, ro = int64_t(row) * w;
  V* slots = reinterpret_cast<V*>(cta);
  V* suf = slots + int64_t(A.wide_max_slots) * w;
  V* pre = suf + int64_t(A.wide_max_suf) * W1;
  // leaf suffix sums (independent of the conditioning value)
  for (int o = 0; o < sb.n_ops; o++) {
    const EstOp op = sh_ops[o];
    const EstIn* in = sh_in + op.in_begin;
    const int p = op.p, m = op.k - (p >= 0 ? 1 : 0);
    for (int a = 0; a < m; a++) {
      const EstIn& x = in[a + (p >= 0 && a >= p ? 1 : 0)];
      if (x.kind != kInLeaf) continue;
      V* sl = suf + int64_t(x.suf) * W1;
      const int32_t* perm = x.perm + ro;
      for (int r = tid; r < w; r += T) sl[r] = ar.from(__ldg(x.msk + ro + __ldg(perm + r)));
      if (tid == 0) sl[w] = ar.zero();
      __syncthreads();
      block_scan_v(ar, sl, w, /*reverse=*/true, sh);
    }
  }
  // conditioned edges: both sketches of each (one per independent cycle), with its ordinal
  const int32_t* cond_s[2 * kEstMaxCond];
  int cond_k[2 * kEstMaxCond];
  int n_cond = 0;
  {
    const EstOp last = sh_ops[sb.n_ops - 1];
    const int n_in = last.in_begin + last.k;
    for (int q = 0; q < n_in && n_cond < 2 * kEstMaxCond; q++)
      if (sh_in[q].kind == kInCond) {
        cond_s[n_cond] = sh_in[q].s + ro;
        cond_k[n_cond++] = sh_in[q].slot;
      }
  }
  V total = ar.zero();
  {
    const EstItem item = A.witems[sb.item_begin + int64_t(row) * sb.n_chunks + ch];
    // a split root: one pass over the root's sorted positions [r_lo, r_hi) of this chunk
    const int c_end = sb.split ? item.c0 + 1 : item.c1;
    const int r_lo = sb.split ? item.c0 : 0, r_hi = sb.split ? item.c1 : w;
    for (int c = item.c0; c < c_end; c++) {
      bool zero = false;
      for (int q = 0; q < n_cond; q++) zero |= __ldg(cond_s[q] + cond_digit(c, cond_k[q], w)) == 0;
      if (zero) continue;  // block-uniform: every merged entry through that table is 0
      for (int o = 0; o < sb.n_ops; o++) {
        const EstOp op = sh_ops[o];
        const EstIn* in = sh_in + op.in_begin;
        const int p = op.p, m = op.k - (p >= 0 ? 1 : 0);
        // 1. suffix sums of messages from non-leaf children, in this table's sorted order
        for (int a = 0; a < m; a++) {
          const EstIn& x = in[a + (p >= 0 && a >= p ? 1 : 0)];
          if (x.kind != kInSlot) continue;
          V* sl = suf + int64_t(x.suf) * W1;
          const V* msg = slots + int64_t(x.slot) * w;
          const int32_t* perm = x.perm + ro;
          for (int r = tid; r < w; r += T) sl[r] = msg[__ldg(perm + r)];
          if (tid == 0) sl[w] = ar.zero();
          __syncthreads();
          block_scan_v(ar, sl, w, /*reverse=*/true, sh);
        }
        // 2a. the conditioned input: |s[c]| and its "attains the minimum" term
        if (tid < m) {
          const EstIn& x = in[tid + (p >= 0 && tid >= p ? 1 : 0)];
          if (x.kind == kInCond) {
            const int32_t v = __ldg(x.s + ro + cond_digit(c, x.slot, w));
            sh_ac[tid] = v < 0 ? uint32_t(-int64_t(v)) : uint32_t(v);
          }
        }
        __syncthreads();
        if (tid < m) {
          const int la = tid + (p >= 0 && tid >= p ? 1 : 0);
          const EstIn& x = in[la];
          if (x.kind == kInCond) {
            const int cx = cond_digit(c, x.slot, w);
            const int rpos = __ldg(wrank_row(x, x, A.d, row, w) + cx);
            const uint32_t tau = sh_ac[tid];
            V v = ar.from(__ldg(x.s + ro + cx));
            for (int b = 0; b < m; b++) {
              if (b == tid) continue;
              const int lb = b + (p >= 0 && b >= p ? 1 : 0);
              const EstIn& y = in[lb];
              if (y.kind == kInCond) {
                if (!(lb < la ? sh_ac[b] > tau : sh_ac[b] >= tau)) v = ar.zero();
              } else {
                const int q = __ldg(wrank_row(x, y, A.d, row, w) + rpos);
                v = ar.mul(v, suf[int64_t(y.suf) * W1 + q]);
              }
            }
            sh_val[tid] = v;
          }
        }
        __syncthreads();
        // 2b. the other inputs: s_l m_l prod_{l' != l, p} G_l'(|s_l|), in l's sorted order
        V root_part = ar.zero();
        for (int a = 0; a < m; a++) {
          const int la = a + (p >= 0 && a >= p ? 1 : 0);
          const EstIn& x = in[la];
          if (x.kind == kInCond) {
            if (p < 0 && tid == 0) root_part = ar.add(root_part, sh_val[a]);
            continue;
          }
          const int32_t* perm = x.perm + ro;
          const uint32_t* absa = x.abs + ro;
          const V* msg = x.kind == kInSlot ? slots + int64_t(x.slot) * w : nullptr;
          V* pl = pre + int64_t(a) * W1;
          const int rb = p < 0 ? r_lo : 0, re = p < 0 ? r_hi : w;  // (a split sub-plan's op is its root)
          for (int r = rb + tid; r < re; r += T) {
            const int j = __ldg(perm + r);
            V v = ar.mul(ar.from(__ldg(x.s + ro + j)), msg ? msg[j] : ar.from(__ldg(x.msk + ro + j)));
            for (int b = 0; b < m; b++) {
              if (b == a) continue;
              const int lb = b + (p >= 0 && b >= p ? 1 : 0);
              const EstIn& y = in[lb];
              if (y.kind == kInCond) {
                const uint32_t tau = __ldg(absa + r);
                if (!(lb < la ? sh_ac[b] > tau : sh_ac[b] >= tau)) v = ar.zero();
              } else {
                v = ar.mul(v, suf[int64_t(y.suf) * W1 + __ldg(wrank_row(x, y, A.d, row, w) + r)]);
              }
            }
            if (p < 0) root_part = ar.add(root_part, v);
            else pl[r + 1] = v;
          }
          if (p >= 0) {
            if (tid == 0) pl[0] = ar.zero();
            __syncthreads();
            block_scan_v(ar, pl + 1, w, /*reverse=*/false, sh);
          }
        }
        if (p < 0) {
          total = ar.add(total, block_sum_v(ar, root_part, sh));
          continue;
        }
        // 3. the message to the parent, in the output sketch's sorted order
        const EstIn& xp = in[p];
        const int32_t* permp = xp.perm + ro;
        const uint32_t* absp = xp.abs + ro;
        V* out = slots + int64_t(op.out_slot) * w;
        for (int r = tid; r < w; r += T) {
          const int jp = __ldg(permp + r);
          const uint32_t tau = __ldg(absp + r);
          V t = ar.from(__ldg(xp.s + ro + jp)), add = ar.zero();
          for (int a = 0; a < m; a++) {
            const int la = a + (a >= p ? 1 : 0);
            const EstIn& x = in[la];
            if (x.kind == kInCond) {
              if (!(la < p ? sh_ac[a] > tau : sh_ac[a] >= tau)) t = ar.zero();
              if (la > p ? sh_ac[a] < tau : sh_ac[a] <= tau) add = ar.add(add, sh_val[a]);
            } else {
              const int q = __ldg(wrank_row(xp, x, A.d, row, w) + r);
              t = ar.mul(t, suf[int64_t(x.suf) * W1 + q]);
              add = ar.add(add, pre[int64_t(a) * W1 + q]);
            }
          }
          out[jp] = ar.add(t, add);
        }
        __syncthreads();
      }
    }
  }
  return total;
}

// Moduli a row needs: the fewest k with B < 2^(62 k - 2) <= P_k / 2 (P_k, the product of the
// first k primes, exceeds 2^(62 k - 1)); 0 when the bound reaches 2^kWideBits or is not finite.
__device__ __forceinline__ int wide_mods_for(double B) {
  if (!(B < ldexp(1.0, kWideBits))) return 0;
  if (B < 1.0) return 1;
  int e;
  frexp(B, &e);  // B < 2^e
  const int k = (e + 2 + 61) / 62;
  return k < 1 ? 1 : (k > kWideMods ? 0 : k);
}

// A queued row's bound: the sum, rounded upwards in unit order, of its units' bounds; for a
// star row on its lattice, |S| times the largest bound of its terms T_a(S \ {a}).
__device__ __forceinline__ double wide_row_bound(const EstArgs& A, uint32_t e) {
  const uint32_t qr = A.wide_queue[4 + e];
  const int nch = wide_row_units(A, qr / uint32_t(A.d));
  const uint64_t* part = A.wide_part + int64_t(A.wide_row_start[e]) * (kWideMods + 1);
  if (uint32_t(A.wide_units[A.wide_row_start[e]]) & kUnitLattice)
    return __dmul_ru(__longlong_as_double((long long)part[kWideMods]),
                     double(__popc(A.subs[qr / uint32_t(A.d)].sbits)));
  double B = 0.0;
  for (int c = 0; c < nch; c++) B = __dadd_ru(B, __longlong_as_double((long long)part[int64_t(c) * (kWideMods + 1) + kWideMods]));
  return B;
}

// Persistent over the units of the queued rows: pass 0 computes every unit's bound, pass 1
// its residues modulo the primes its row needs (the others are skipped).
__global__ void __launch_bounds__(kWideThreads, kWideCtasPerSm) k_estimate_wide(const __grid_constant__ EstArgs A, int pass) {
  __shared__ EstOp sh_ops[kEstMaxOps];
  __shared__ EstIn sh_in[kEstMaxSubIn];
  __shared__ uint64_t sh_u[33];
  __shared__ double sh_d[33];
  __shared__ uint64_t sh_valu[CMP_MAX_SKETCHES];
  __shared__ double sh_vald[CMP_MAX_SKETCHES];
  __shared__ uint32_t sh_ac[CMP_MAX_SKETCHES];
  const uint32_t n_units = min(A.wide_queue[2], uint32_t(A.wide_unit_cap));
  const int per_unit = pass == 0 ? 1 : kWideMods;
  const int64_t jobs = int64_t(n_units) * per_unit;
  unsigned char* cta = static_cast<unsigned char*>(A.wide_scratch) + int64_t(blockIdx.x) * A.wide_scratch_per_cta;
  for (int64_t g = blockIdx.x; g < jobs; g += gridDim.x) {
    const int64_t u = g / per_unit;
    const int j = pass == 0 ? kWideMods : int(g % per_unit);
    const uint64_t ent = A.wide_units[u];
    if (ent == ~0ull) continue;  // taken by a row that did not fit (its sub-plan is reported NaN)
    if (uint32_t(ent) & kUnitLattice) continue;  // filled by its star family's lattice
    const uint32_t e = uint32_t(ent >> 32);
    const int ch = int(uint32_t(ent));
    if (pass == 1 && j >= wide_mods_for(wide_row_bound(A, e))) continue;  // block-uniform
    const uint32_t qr = A.wide_queue[4 + e];
    const int64_t q = qr / uint32_t(A.d);
    const int row = int(qr % uint32_t(A.d));
    const EstSub sb = A.wsubs[q];
    uint64_t result = 0;
    if (sb.single) {  // never queued (an exact count); kept for completeness
      const int64_t n = *sb.sv;
      result = j < kWideMods ? ModArith{wide_p(j), wide_c(j)}.from(n)
                             : uint64_t(__double_as_longlong(fabs(double(n))));
    } else if (sb.n_ops > 0) {
      const int in0 = A.wops[sb.op_begin].in_begin;
      const EstOp last = A.wops[sb.op_begin + sb.n_ops - 1];
      const int n_in = last.in_begin + last.k - in0;
      for (int o = threadIdx.x; o < sb.n_ops; o += blockDim.x) {
        EstOp op = A.wops[sb.op_begin + o];
        op.in_begin -= in0;
        sh_ops[o] = op;
      }
      for (int k = threadIdx.x; k < n_in; k += blockDim.x) sh_in[k] = A.winputs[in0 + k];
      __syncthreads();
      if (j < kWideMods) {
        const ModArith ar{wide_p(j), wide_c(j)};
        result = wide_row(ar, A, sb, row, ch, sh_ops, sh_in, sh_u, sh_valu, sh_ac, cta);
      } else {
        const BoundArith ar{};
        result =
            uint64_t(__double_as_longlong(wide_row(ar, A, sb, row, ch, sh_ops, sh_in, sh_d, sh_vald, sh_ac, cta)));
      }
    }
    if (threadIdx.x == 0) A.wide_part[u * (kWideMods + 1) + j] = result;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- star rows on the lattice
// A queued star row S of family f and sketch row i has E_i(S) = sum_{a in S} T_a(S \ {a})
// (the family's lattice, estimate_star.cu).  When the (family, row) has enough queued rows
// that one lattice per modulus costs less than their generic contractions (K 2^(K-1)
// multiply-adds per sorted position against about |S|^2 / 4 gathered products per row,
// weighted 3 for the gathers), the family's lattice is evaluated again modulo each prime the
// rows need and as a magnitude bound, and every entry T_a(V) whose leaf set V + {a} is a
// queued row is added to that row's unit: its residue modulo p_j (an exact modular sum,
// whatever the order) and its bound (the unit keeps the largest; the row's bound is |S|
// times it).  Otherwise the row's unit runs the generic contraction.

// Per queued star row: the route of its (family, row), taken from the count of its rows.
__global__ void k_star_route(const __grid_constant__ EstArgs A) {
  const uint32_t n_rows = min(A.wide_queue[0], uint32_t(A.wide_qcap));
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_rows || A.wide_row_start[e] < 0) return;
  const uint32_t qr = A.wide_queue[4 + e];
  const int64_t q = qr / uint32_t(A.d);
  const int row = int(qr % uint32_t(A.d));
  if (!wide_star_row(A, q)) return;
  const int32_t f = A.subs[q].star;
  const int K = A.star[f].K;
  const int64_t fr = int64_t(f) * A.d + row;
  const uint64_t cnt = A.wide_star_cnt[fr];
  if (cnt * uint64_t(3 * K) >= (uint64_t(1) << (K + 1))) {
    A.wide_star_on[fr] = 1;
    return;
  }
  A.wide_units[A.wide_row_start[e]] = uint64_t(e) << 32;  // chunk 0 of its generic (tree) plan
}

// Per queued star row on a lattice: the most primes a row of its (family, row) needs.
__global__ void k_star_kmax(const __grid_constant__ EstArgs A) {
  const uint32_t n_rows = min(A.wide_queue[0], uint32_t(A.wide_qcap));
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_rows || A.wide_row_start[e] < 0) return;
  if (!(uint32_t(A.wide_units[A.wide_row_start[e]]) & kUnitLattice)) return;
  const uint32_t qr = A.wide_queue[4 + e];
  const int64_t q = qr / uint32_t(A.d);
  atomicMax(A.wide_star_kmax + int64_t(A.subs[q].star) * A.d + int(qr % uint32_t(A.d)),
            wide_mods_for(wide_row_bound(A, e)));
}

template <class M>
__device__ __forceinline__ M star_arith(int j);
template <>
__device__ __forceinline__ ModArith star_arith<ModArith>(int j) {
  return ModArith{wide_p(j), wide_c(j)};
}
template <>
__device__ __forceinline__ BoundArith star_arith<BoundArith>(int) {
  return BoundArith{};
}

// The lattice units of the families with rows on their lattice, in arithmetic M: pass 0 the
// magnitude bounds (M = BoundArith), pass 1 the residues modulo the primes their rows need
// (one unit per prime).  The layout of a unit follows k_star_lattice: 2^m1 A-side subsets
// (the block's high bits fixed) times 2^k2 B-side subsets, entries split over the threads,
// sorted positions in chunks of kStarR.
template <class M>
__global__ void __launch_bounds__(kStarThreads) k_star_wide(const __grid_constant__ EstArgs A, int pass) {
  using V = typename M::V;
  constexpr int R = kStarR, NB = 1 << kStarMaxK2;
  __shared__ V Bs[R * NB];
  __shared__ V As[R * 16];
  __shared__ V red[kStarThreads];
  __shared__ V fv[(CMP_MAX_SKETCHES - 1) * R];
  __shared__ V wv[R];
  const int tid = threadIdx.x, w = A.w, d = A.d;
  const int per = pass == 0 ? 1 : kWideMods;
  const int64_t n_lat = A.n_star_units - A.n_star_suf_units;
  for (int64_t g = blockIdx.x; g < n_lat * per; g += gridDim.x) {
    const StarUnit u = A.star_units[A.n_star_suf_units + g / per];
    const int j = pass == 0 ? kWideMods : int(g % per);
    const int64_t fr = int64_t(u.fam) * d + u.row;
    if (!A.wide_star_on[fr]) continue;  // block-uniform
    if (pass == 1 && j >= A.wide_star_kmax[fr]) continue;
    const M ar = star_arith<M>(j);
    const StarFam F = A.star[u.fam];
    const int K = F.K, k = K - 1, k1 = F.k1, k2 = F.k2, m1 = F.m1;
    const int NV2 = 1 << k2, E = 1 << (m1 + k2);
    const int Ep = E < kStarThreads ? E : kStarThreads;
    const int L = kStarThreads / Ep, J = E / Ep;
    const int es = tid % Ep, lane = tid / Ep;
    const int64_t ro = int64_t(u.row) * w;
    const EstIn xa = A.inputs[F.in_begin + u.a];
    const int64_t* suf0 = A.star_suf + F.suf_off + int64_t(u.row) * K * (int64_t(w) + 1);
    V acc[16];
#pragma unroll
    for (int q = 0; q < 16; q++) acc[q] = ar.zero();
    for (int r0 = 0; r0 < w; r0 += R) {
      // 1. the chunk's factors f[b][r] (position b of U \ {a}) and w[r]
      for (int q = tid; q < (k + 1) * R; q += kStarThreads) {
        const int b = q / R, rr = q % R, r = r0 + rr;
        if (b < k) {
          V f = ar.zero();
          if (r < w) {
            const int ub = b < u.a ? b : b + 1;
            const EstIn& xb = A.inputs[F.in_begin + ub];
            const int32_t pos = __ldg(xa.rk + (int64_t(xb.tslot) * d + u.row) * w + r);
            f = ar.from(suf0[int64_t(ub) * (w + 1) + pos]);  // |suffix sum| < 2^51
          }
          fv[b * R + rr] = f;
        } else {
          V wr = ar.zero();
          if (r < w) {
            const int32_t jj = __ldg(xa.perm + ro + r);
            wr = ar.from_wide(int64_t(__ldg(xa.s + ro + jj)) * int64_t(__ldg(xa.msk + ro + jj)));
          }
          wv[rr] = wr;
        }
      }
      __syncthreads();
      // 2. table roots: B[r][0] = 1, A[r][0] = w(r) times the factors of the block's bits
      for (int rr = tid; rr < R; rr += kStarThreads) {
        Bs[rr * NB] = ar.one();
        V v = wv[rr];
        for (int i = 0; i < k1 - m1; i++)
          if ((u.blk >> i) & 1) v = ar.mul(v, fv[(m1 + i) * R + rr]);
        As[rr * 16] = v;
      }
      __syncthreads();
      // 3. doubling: entries [h, 2h) from [0, h) times the factor of bit jj
      const int steps = k2 > m1 ? k2 : m1;
      for (int jj = 0; jj < steps; jj++) {
        const int h = 1 << jj;
        if (jj < k2)
          for (int q = tid; q < h * R; q += kStarThreads) {
            const int rr = q / h, idx = h + q % h;
            Bs[rr * NB + idx] = ar.mul(Bs[rr * NB + idx - h], fv[(k1 + jj) * R + rr]);
          }
        if (jj < m1)
          for (int q = tid; q < h * R; q += kStarThreads) {
            const int rr = q / h, idx = h + q % h;
            As[rr * 16 + idx] = ar.mul(As[rr * 16 + idx - h], fv[jj * R + rr]);
          }
        __syncthreads();
      }
      // 4. multiply-add over the chunk's positions (residues: the at most kStarR products of
      //    a lane summed exactly in 128 bits, below 2^128, then reduced once)
#pragma unroll
      for (int q = 0; q < 16; q++) {
        if (q >= J) break;
        const int e = es + Ep * q;
        const int v1 = e >> k2, v2 = e & (NV2 - 1);
        if constexpr (std::is_same<M, ModArith>::value) {
          u128 s = 0;
          for (int rr = lane; rr < R; rr += L) s += u128(As[rr * 16 + v1]) * Bs[rr * NB + v2];
          acc[q] = ar.add(acc[q], ar.reduce128(s));
        } else {
          V s = acc[q];
          for (int rr = lane; rr < R; rr += L) s = ar.add(s, ar.mul(As[rr * 16 + v1], Bs[rr * NB + v2]));
          acc[q] = s;
        }
      }
      __syncthreads();
    }
    // 5. lanes of one entry (L > 1 means J = 1): their sum
    if (L > 1) {
      red[tid] = acc[0];
      __syncthreads();
      if (lane == 0) {
        V s = ar.zero();
        for (int l = 0; l < L; l++) s = ar.add(s, red[es + Ep * l]);
        acc[0] = s;
      }
      __syncthreads();
    }
    // 6. each entry T_a(V) to the unit of the queued row V + {a}, if there is one
    if (lane == 0) {
      const uint32_t n_rows = min(A.wide_queue[0], uint32_t(A.wide_qcap));
#pragma unroll
      for (int q = 0; q < 16; q++) {
        if (q >= J) break;
        const int e = es + Ep * q;
        const int v1 = e >> k2, v2 = e & (NV2 - 1);
        const uint32_t Vb = uint32_t((u.blk << m1) | v1) | (uint32_t(v2) << k1);
        const uint32_t low = (1u << u.a) - 1u;
        const uint32_t S = ((Vb & ~low) << 1) | (1u << u.a) | (Vb & low);
        const int32_t sq = A.star_q[F.q_off + S];
        if (sq < 0) continue;
        const int64_t rq = int64_t(sq) * d + u.row;
        const int32_t slot = A.wide_slot[rq];  // stale unless the row was queued by this call:
        if (slot < 0 || uint32_t(slot) >= n_rows || A.wide_row_start[slot] < 0 ||
            A.wide_queue[4 + slot] != uint32_t(rq))
          continue;  // the queue entry decides
        const int64_t unit = A.wide_row_start[slot];
        if (!(uint32_t(A.wide_units[unit]) & kUnitLattice)) continue;
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(A.wide_part + unit * (kWideMods + 1) + j);
        if constexpr (std::is_same<V, double>::value) {
          atomicMax(dst, (unsigned long long)__double_as_longlong(acc[q]));  // >= 0: bits order as values
        } else {
          const uint64_t p = wide_p(j);
          unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(dst), seen = ~0ull;
          // (old + v) mod p, both below p < 2^62; a failed exchange means another leaf's add
          // landed (at most |S| - 1 of them), so the bound is never reached
          for (int tries = 0; tries < 1024 && old != seen; tries++) {
            seen = old;
            const uint64_t s = uint64_t(seen) + acc[q];
            old = atomicCAS(dst, seen, (unsigned long long)(s >= p ? s - p : s));
          }
          if (old != seen) set_status(A.status, CMP_ETIMEOUT);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- wide integers
// Signed values as sign + kWideLimbs little-endian 64-bit limbs of the magnitude.
struct Wide {
  uint64_t m[kWideLimbs];
  int neg;
};

__device__ __forceinline__ int wide_cmp_mag(const uint64_t* a, const uint64_t* b) {
  for (int k = kWideLimbs - 1; k >= 0; k--)
    if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
  return 0;
}
__device__ __forceinline__ bool wide_less(const Wide& a, const Wide& b) {
  const bool az = wide_cmp_mag(a.m, b.m) == 0 && a.neg == b.neg;
  if (az) return false;
  if (a.neg != b.neg) return a.neg;  // a negative, b not (zero is never negative here)
  const int c = wide_cmp_mag(a.m, b.m);
  return a.neg ? c > 0 : c < 0;
}

// Round-to-nearest-even of (neg ? -1 : 1) * (top 2^(64 kWideLimbs) + mag) to double, from
// the definition: the leading 53 bits, then the half-ulp and sticky bits.
__device__ double wide_mag_to_double(bool neg, uint32_t top, const uint64_t* mag) {
  int hi = kWideLimbs - 1;
  while (hi >= 0 && mag[hi] == 0) hi--;
  if (top == 0 && hi < 0) return 0.0;
  // bit length of the value
  const int nb = top ? 64 * kWideLimbs + 1 : 64 * hi + (64 - __clzll(mag[hi]));
  auto bit = [&](int k) -> uint64_t {  // bit k of the value
    if (k >= 64 * kWideLimbs) return top;
    return (mag[k >> 6] >> (k & 63)) & 1ull;
  };
  double r;
  if (nb <= 53) {
    r = double(mag[0]);
  } else {
    const int sh = nb - 53;
    uint64_t s = 0;
    for (int k = nb - 1; k >= sh; k--) s = (s << 1) | bit(k);
    const uint64_t half = bit(sh - 1);
    bool sticky = false;
    for (int k = 0; k < sh - 1 && !sticky; k++) sticky = bit(k) != 0;
    if (half && (sticky || (s & 1))) s++;
    int e = sh;
    if (s == (1ull << 53)) {
      s >>= 1;
      e++;
    }
    r = ldexp(double(s), e);
  }
  return neg ? -r : r;
}

__device__ __forceinline__ uint64_t mulmod_p(uint64_t a, uint64_t b, int j) {
  const ModArith ar{wide_p(j), wide_c(j)};
  return ar.mul(a, b);
}
__device__ uint64_t powmod_p(uint64_t a, uint64_t e, int j) {
  uint64_t r = 1, b = a;
  while (e) {
    if (e & 1) r = mulmod_p(r, b, j);
    b = mulmod_p(b, b, j);
    e >>= 1;
  }
  return r;
}

constexpr int kWideFinThreads = 128;

}  // namespace

// One CTA per queued sub-plan (persistent), thread i < d takes row i: its int128 value when
// it stayed in range, else the integer rebuilt from its residues by Garner's algorithm;
// thread 0 takes the exact median and rounds it once.
__global__ void __launch_bounds__(kWideFinThreads) k_estimate_wide_finalize(const __grid_constant__ EstArgs A,
                                                                             double* __restrict__ est,
                                                                             int64_t* __restrict__ wide_rows) {
  __shared__ uint64_t inv[kWideMods][kWideMods];          // inv[i][j] = p_i^-1 mod p_j, i < j
  __shared__ uint64_t Pk[kWideMods + 1][kWideLimbs + 1];  // Pk[k] = p_0 ... p_{k-1}
  __shared__ Wide rows[CMP_MAX_D];
  __shared__ int32_t bad;
  const uint32_t n_sub_q = A.wide_queue[1];
  if (n_sub_q == 0 || blockIdx.x >= n_sub_q) return;
  const int tid = threadIdx.x, d = A.d;
  for (int t = tid; t < kWideMods * kWideMods; t += blockDim.x) {
    const int i = t / kWideMods, j = t % kWideMods;
    if (i < j) inv[i][j] = powmod_p(wide_p(i) % wide_p(j), wide_p(j) - 2, j);  // Fermat: p_j is prime
  }
  if (tid == 0) {
    for (int l = 0; l <= kWideLimbs; l++) Pk[0][l] = l == 0 ? 1 : 0;
    for (int k = 1; k <= kWideMods; k++) {  // Pk[k] = Pk[k-1] p_{k-1}
      uint64_t carry = 0;
      for (int l = 0; l <= kWideLimbs; l++) {
        const u128 t = u128(Pk[k - 1][l]) * wide_p(k - 1) + carry;
        Pk[k][l] = uint64_t(t);
        carry = uint64_t(t >> 64);
      }
    }
  }
  __syncthreads();
  for (uint32_t k = blockIdx.x; k < n_sub_q; k += gridDim.x) {
    const int64_t q = A.wide_queue[4 + A.wide_qcap + k];
    if (tid == 0) bad = 0;
    __syncthreads();
    if (tid < d) {
      const int32_t slot = A.wide_slot[q * d + tid];
      Wide wv;
      if (slot < 0) {  // in range: the int128 row
        const i128 v = A.wide_in[q * d + tid];
        wv.neg = v < 0 ? 1 : 0;
        const u128 m = v < 0 ? u128(0) - u128(v) : u128(v);
        for (int l = 0; l < kWideLimbs; l++) wv.m[l] = l == 0 ? uint64_t(m) : (l == 1 ? uint64_t(m >> 64) : 0);
      } else {
        const int K = wide_mods_for(wide_row_bound(A, uint32_t(slot)));
        if (K == 0) atomicOr(&bad, 1);
        // the row's residues: its units' residues summed modulo each prime
        const int nch = wide_row_units(A, q);
        const uint64_t* part = A.wide_part + int64_t(A.wide_row_start[slot]) * (kWideMods + 1);
        uint64_t r[kWideMods];
        for (int j = 0; j < K; j++) {
          const uint64_t pj = wide_p(j);
          uint64_t s = 0;
          for (int c = 0; c < nch; c++) {
            s += part[int64_t(c) * (kWideMods + 1) + j];  // both < p_j < 2^62: no wrap
            s = s >= pj ? s - pj : s;
          }
          r[j] = s;
        }
        // Garner: x = v_0 + v_1 p_0 + v_2 p_0 p_1 + ..., v_j from the residue mod p_j
        uint64_t v[kWideMods];
        for (int j = 0; j < K; j++) {
          const uint64_t pj = wide_p(j);
          uint64_t t = r[j];
          for (int i = 0; i < j; i++) {
            const uint64_t vi = v[i] >= pj ? v[i] - pj : v[i];
            t = t >= vi ? t - vi : t + pj - vi;
            t = mulmod_p(t, inv[i][j], j);
          }
          v[j] = t;
        }
        uint64_t x[kWideLimbs + 1];
        for (int l = 0; l <= kWideLimbs; l++) x[l] = 0;
        for (int j = K - 1; j >= 0; j--) {  // x = x p_j + v_j
          uint64_t carry = v[j];
          for (int l = 0; l <= kWideLimbs; l++) {
            const u128 t = u128(x[l]) * wide_p(j) + carry;
            x[l] = uint64_t(t);
            carry = uint64_t(t >> 64);
          }
        }
        // x in [0, P_K): E = x when x < P_K - x, else E = -(P_K - x)
        uint64_t y[kWideLimbs + 1];
        uint64_t borrow = 0;
        for (int l = 0; l <= kWideLimbs; l++) {
          const u128 t = u128(Pk[K][l]) - x[l] - borrow;
          y[l] = uint64_t(t);
          borrow = (t >> 64) ? 1 : 0;
        }
        bool x_small = true;
        for (int l = kWideLimbs; l >= 0; l--)
          if (x[l] != y[l]) {
            x_small = x[l] < y[l];
            break;
          }
        wv.neg = x_small ? 0 : 1;
        for (int l = 0; l < kWideLimbs; l++) wv.m[l] = x_small ? x[l] : y[l];
        bool zero = true;
        for (int l = 0; l < kWideLimbs; l++) zero &= wv.m[l] == 0;
        if (zero) wv.neg = 0;
      }
      rows[tid] = wv;
      if (wide_rows) {  // two's complement limbs
        int64_t* o = wide_rows + (q * d + tid) * kWideLimbs;
        uint64_t c = 1;
        for (int l = 0; l < kWideLimbs; l++) {
          uint64_t limb = wv.m[l];
          if (wv.neg) {
            const u128 t = u128(~limb) + c;
            limb = uint64_t(t);
            c = uint64_t(t >> 64);
          }
          o[l] = int64_t(limb);
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      const EstSub sb = A.subs[q];
      if (bad) {
        est[q] = __longlong_as_double(0x7ff8000000000000ll);
        set_status(A.status, CMP_EOVERFLOW);
      } else {
        for (int a = 1; a < d; a++) {  // insertion sort of exact integers
          const Wide v = rows[a];
          int b = a - 1;
          while (b >= 0 && wide_less(v, rows[b])) {
            rows[b + 1] = rows[b];
            b--;
          }
          rows[b + 1] = v;
        }
        double med;
        if (d & 1) {
          med = wide_mag_to_double(rows[d / 2].neg, 0, rows[d / 2].m);
        } else {  // exact (a + b) / 2: signed sum, then one rounding
          const Wide& a = rows[d / 2 - 1];
          const Wide& b = rows[d / 2];
          uint64_t s[kWideLimbs];
          uint32_t top = 0;
          bool neg;
          if (a.neg == b.neg) {
            uint64_t c = 0;
            for (int l = 0; l < kWideLimbs; l++) {
              const u128 t = u128(a.m[l]) + b.m[l] + c;
              s[l] = uint64_t(t);
              c = uint64_t(t >> 64);
            }
            top = uint32_t(c);
            neg = a.neg;
          } else {
            const bool a_big = wide_cmp_mag(a.m, b.m) >= 0;
            const uint64_t* big = a_big ? a.m : b.m;
            const uint64_t* small = a_big ? b.m : a.m;
            uint64_t br = 0;
            for (int l = 0; l < kWideLimbs; l++) {
              const u128 t = u128(big[l]) - small[l] - br;
              s[l] = uint64_t(t);
              br = (t >> 64) ? 1 : 0;
            }
            neg = a_big ? a.neg : b.neg;
          }
          med = wide_mag_to_double(neg, top, s) * 0.5;
        }
        est[q] = __dmul_rn(med, sb.scale);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_estimate_wide(const EstArgs& a, double* est, int64_t* wide_rows, cudaStream_t st) {
  if (!a.wide) return cudaSuccess;
  // star rows on their families' lattices (only when the plan has lattice units)
  const bool lat = a.n_star_units > a.n_star_suf_units;
  const unsigned row_blocks = unsigned((a.wide_qcap + 255) / 256);
  const unsigned lat_grid =
      unsigned(std::min<int64_t>(int64_t(sm_count()) * 4, (a.n_star_units - a.n_star_suf_units) * kWideMods));
  if (lat) {
    k_star_route<<<row_blocks, 256, 0, st>>>(a);
    k_star_wide<BoundArith><<<lat_grid, kStarThreads, 0, st>>>(a, 0);
  }
  k_estimate_wide<<<unsigned(a.wide_grid), kWideThreads, 0, st>>>(a, 0);  // bounds
  if (lat) {
    k_star_kmax<<<row_blocks, 256, 0, st>>>(a);
    k_star_wide<ModArith><<<lat_grid, kStarThreads, 0, st>>>(a, 1);
  }
  k_estimate_wide<<<unsigned(a.wide_grid), kWideThreads, 0, st>>>(a, 1);  // residues
  k_estimate_wide_finalize<<<unsigned(sm_count()), kWideFinThreads, 0, st>>>(a, est, wide_rows);
  return cudaGetLastError();
}

}  // namespace cmpk
