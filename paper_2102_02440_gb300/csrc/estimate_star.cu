// Star families of the estimate: every sub-plan made of one root table joined to leaves,
// for all leaf subsets of one (graph, root) at once (Sec. 5: products of sketches cached
// across the sub-plans of an enumeration; Sec. 4.2: the merged root sketch contracted with
// the leaf sketches).
//
// With the root's sketches on its leaf edges U (ascending id), a star over leaf set S has,
// in sketch row i, the exact row estimate
//   E(S) = sum_{a in S} sum_r w_a(r) prod_{b in S, b != a} f_ab(r),
// where r runs over a's sorted order (the merged entry takes a's value where a's |value|
// is the minimum), w_a(r) = s_a[pi_a(r)] m_a[pi_a(r)] (root sketch times leaf sketch) and
// f_ab(r) is the suffix sum of leaf b's sketch in b's sorted order from the cross rank of
// a's position r.  The factors f_ab(r) do not depend on S, so the sums
//   T_a(V) = sum_r w_a(r) prod_{b in V} f_ab(r)   for every V in U \ {a}
// are a product of two tables over r: A[V1][r] = w_a(r) prod_{V1} f (the k1 low positions)
// and B[V2][r] = prod_{V2} f (the k2 high positions), T_a(V1 | V2 << k1) = sum_r A B.  Each
// table entry is built from a smaller one by one multiplication, each T entry costs one
// multiply-add per r, and E(S) is a gather of |S| entries (k_estimate_finalize).
//
// Every value is an exact int128.  A table entry whose exact value leaves int128 is flagged
// (it stays flagged through further nonzero factors; a zero factor makes it an exact 0); a
// T entry is flagged when one of its terms or partial sums leaves int128, and the gather
// flags the row, so a row that is not flagged is exact.
#include <cuda_runtime.h>

#include <algorithm>

#include "est_arith.cuh"

namespace cmpk {
namespace {

__device__ __forceinline__ const int32_t* star_rank_row(const EstIn& x, const EstIn& y, int d, int row, int w) {
  return x.rk + (int64_t(y.tslot) * d + row) * w;
}

// An upper bound of |v| in float (+inf for an out-of-range entry): the high word plus one,
// or the low word, rounded up.
__device__ __forceinline__ float star_mag(i128 v, bool fl) {
  if (fl) return __int_as_float(0x7f800000);
  const u128 m = v < 0 ? u128(0) - u128(v) : u128(v);
  const uint64_t hi = uint64_t(m >> 64);
  return hi ? __ull2float_ru(hi + 1) * 0x1p64f : __ull2float_ru(uint64_t(m));
}

// v *= f with the out-of-range flag carried (see the file comment).
__device__ __forceinline__ void star_step(i128& v, bool& fl, int64_t f) {
  if (f == 0) {
    v = 0;
    fl = false;
  } else if (!fl) {
    fl = mul_ovf(v, i128(f), &v);
  }
}

// One CTA per (family, row, leaf b): b's suffix sums in b's sorted order, [w + 1] int64
// (|m| < 2^31 and w <= 2^20: no overflow).
__global__ void __launch_bounds__(kStarThreads) k_star_suf(const __grid_constant__ EstArgs A) {
  __shared__ i128 sh_i128[33];
  __shared__ int32_t sh_flag[1];
  BlockScratch bs{sh_i128, sh_flag};
  const StarUnit u = A.star_units[blockIdx.x];
  const StarFam F = A.star[u.fam];
  const EstIn x = A.inputs[F.in_begin + u.a];
  const int w = A.w;
  const int64_t ro = int64_t(u.row) * w;
  int64_t* sl = A.star_suf + F.suf_off + (int64_t(u.row) * F.K + u.a) * (int64_t(w) + 1);
  for (int r = threadIdx.x; r < w; r += blockDim.x) sl[r] = int64_t(__ldg(x.msk + ro + __ldg(x.perm + ro + r)));
  if (threadIdx.x == 0) {
    sl[w] = 0;
    sh_flag[0] = 0;
  }
  __syncthreads();
  block_scan(sl, w, /*reverse=*/true, bs);
}

// Lattice units (family, row, a, blk), persistent over the unit list.  A unit computes
// T_a(V) for the 2^m1 A-side subsets of block blk (bits m1..k1-1 of V1 = blk) and all 2^k2
// B-side subsets: E = 2^(m1+k2) entries, Ep = min(E, 256) entry slots, L = 256 / Ep lanes
// per slot splitting the sorted positions (reduced at the end), J = E / Ep entries per
// thread.  Shared memory per chunk of kStarR positions: B[r][v2], A[r][v1] (int128 with byte
// flags), the factors f[j][r] and w[r].
__global__ void __launch_bounds__(kStarThreads) k_star_lattice(const __grid_constant__ EstArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int R = kStarR, NB = 1 << kStarMaxK2;
  i128* Bs = reinterpret_cast<i128*>(smem);                      // [R][256]
  i128* As = Bs + R * NB;                                          // [R][16]
  i128* red = As + R * 16;                                         // [256]
  int64_t* fv = reinterpret_cast<int64_t*>(red + kStarThreads);  // [15][R]
  int64_t* wv = fv + 15 * R;                                       // [R]
  uint8_t* Bf = reinterpret_cast<uint8_t*>(wv + R);               // [R][256]
  uint8_t* Af = Bf + R * NB;                                       // [R][16]
  uint8_t* redf = Af + R * 16;                                     // [256]
  float* Bm = reinterpret_cast<float*>(redf + kStarThreads);      // [R][256] magnitude bounds
  float* Am = Bm + R * NB;                                         // [R][16]
  const int tid = threadIdx.x;
  const int w = A.w, d = A.d;
  for (int64_t ui = A.n_star_suf_units + blockIdx.x; ui < A.n_star_units; ui += gridDim.x) {
    const StarUnit u = A.star_units[ui];
    const StarFam F = A.star[u.fam];
    const int K = F.K, k = K - 1, k1 = F.k1, k2 = F.k2, m1 = F.m1;
    const int NV2 = 1 << k2, E = 1 << (m1 + k2);
    const int Ep = E < kStarThreads ? E : kStarThreads;
    const int L = kStarThreads / Ep, J = E / Ep;
    const int es = tid % Ep, lane = tid / Ep;
    const int64_t ro = int64_t(u.row) * w;
    const EstIn xa = A.inputs[F.in_begin + u.a];
    const int64_t* suf0 = A.star_suf + F.suf_off + int64_t(u.row) * K * (int64_t(w) + 1);
    i128 acc[16];
    uint32_t accf = 0;
#pragma unroll
    for (int j = 0; j < 16; j++) acc[j] = 0;

    for (int r0 = 0; r0 < w; r0 += R) {
      // 1. the chunk's factors f[j][r] (position j of U \ {a}) and w[r]
      for (int q = tid; q < (k + 1) * R; q += kStarThreads) {
        const int j = q / R, rr = q % R, r = r0 + rr;
        if (j < k) {
          int64_t f = 0;
          if (r < w) {
            const int ub = j < u.a ? j : j + 1;
            const EstIn& xb = A.inputs[F.in_begin + ub];
            const int32_t pos = __ldg(star_rank_row(xa, xb, d, u.row, w) + r);
            f = suf0[int64_t(ub) * (w + 1) + pos];
          }
          fv[j * R + rr] = f;
        } else {
          int64_t wr = 0;
          if (r < w) {
            const int32_t jj = __ldg(xa.perm + ro + r);
            wr = int64_t(__ldg(xa.s + ro + jj)) * int64_t(__ldg(xa.msk + ro + jj));  // |int32 int32| < 2^62
          }
          wv[rr] = wr;
        }
      }
      __syncthreads();
      // 2. table roots: B[r][0] = 1, A[r][0] = w(r) times the factors of blk's bits
      for (int rr = tid; rr < R; rr += kStarThreads) {
        Bs[rr * NB] = 1;
        Bf[rr * NB] = 0;
        Bm[rr * NB] = 1.0f;
        i128 v = i128(wv[rr]);
        bool fl = false;
        for (int i = 0; i < k1 - m1; i++)
          if ((u.blk >> i) & 1) star_step(v, fl, fv[(m1 + i) * R + rr]);
        As[rr * 16] = v;
        Af[rr * 16] = fl;
        Am[rr * 16] = star_mag(v, fl);
      }
      __syncthreads();
      // 3. doubling: entries [h, 2h) from [0, h) times the factor of bit jj
      const int steps = k2 > m1 ? k2 : m1;
      for (int jj = 0; jj < steps; jj++) {
        const int h = 1 << jj;
        if (jj < k2)
          for (int q = tid; q < h * R; q += kStarThreads) {
            const int rr = q / h, idx = h + q % h;
            i128 v = Bs[rr * NB + idx - h];
            bool fl = Bf[rr * NB + idx - h];
            star_step(v, fl, fv[(k1 + jj) * R + rr]);
            Bs[rr * NB + idx] = v;
            Bf[rr * NB + idx] = fl;
            Bm[rr * NB + idx] = star_mag(v, fl);
          }
        if (jj < m1)
          for (int q = tid; q < h * R; q += kStarThreads) {
            const int rr = q / h, idx = h + q % h;
            i128 v = As[rr * 16 + idx - h];
            bool fl = Af[rr * 16 + idx - h];
            star_step(v, fl, fv[jj * R + rr]);
            As[rr * 16 + idx] = v;
            Af[rr * 16 + idx] = fl;
            Am[rr * 16 + idx] = star_mag(v, fl);
          }
        __syncthreads();
      }
      // 4. multiply-add over the chunk's positions.  When the magnitude bounds keep the product
      //    below 2^126 (float rounding stays far from 2^127), the product modulo 2^128 is exact.
#pragma unroll
      for (int j = 0; j < 16; j++) {
        if (j >= J) break;
        const int e = es + Ep * j;
        const int v1 = e >> k2, v2 = e & (NV2 - 1);
        i128 s = acc[j];
        bool sf = (accf >> j) & 1u;
        for (int rr = lane; rr < R; rr += L) {
          const i128 a = As[rr * 16 + v1], b = Bs[rr * NB + v2];
          if (Am[rr * 16 + v1] * Bm[rr * NB + v2] < 0x1p126f) {
            sf |= add_ovf(s, i128(u128(a) * u128(b)), &s);
            continue;
          }
          const bool fa = Af[rr * 16 + v1], fb = Bf[rr * NB + v2];
          if ((!fa && a == 0) || (!fb && b == 0)) continue;  // an exact zero factor
          if (fa || fb) {
            sf = true;
            continue;
          }
          i128 p;
          sf |= mul_ovf(a, b, &p);
          sf |= add_ovf(s, p, &s);
        }
        acc[j] = s;
        accf = (accf & ~(1u << j)) | (uint32_t(sf) << j);
      }
      __syncthreads();
    }
    // 5. lanes of one slot (L > 1 means J = 1): exact sum of their partial sums
    if (L > 1) {
      red[tid] = acc[0];
      redf[tid] = uint8_t(accf & 1u);
      __syncthreads();
      if (lane == 0) {
        i128 s = 0;
        bool sf = false;
        for (int l = 0; l < L; l++) {
          const int t = es + Ep * l;
          if (redf[t]) sf = true;
          else sf |= add_ovf(s, red[t], &s);
        }
        acc[0] = s;
        accf = sf ? 1u : 0u;
      }
      __syncthreads();
    }
    if (lane == 0) {
      const int64_t base = F.t_off + ((int64_t(u.row) * K + u.a) << k);
#pragma unroll
      for (int j = 0; j < 16; j++) {
        if (j >= J) break;
        const int e = es + Ep * j;
        const int v1 = e >> k2, v2 = e & (NV2 - 1);
        const int64_t V = int64_t((u.blk << m1) | v1) | (int64_t(v2) << k1);
        A.star_t[base + V] = acc[j];
        A.star_tf[base + V] = uint8_t((accf >> j) & 1u);
      }
    }
  }
}

}  // namespace

cudaError_t launch_estimate_star(const EstArgs& a, cudaStream_t st) {
  if (a.n_star_units <= 0) return cudaSuccess;
  if (a.n_star_suf_units > 0) k_star_suf<<<unsigned(a.n_star_suf_units), kStarThreads, 0, st>>>(a);
  const int64_t lat = a.n_star_units - a.n_star_suf_units;
  if (lat > 0) {
    const size_t smem = star_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_star_lattice, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(lat, int64_t(sm_count()) * 2);  // two 80 KB CTAs per SM
    k_star_lattice<<<unsigned(grid), kStarThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace cmpk
