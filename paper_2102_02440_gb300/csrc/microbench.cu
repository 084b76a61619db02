// Microbenchmark of the Carter-Wegman arithmetic of the build (the integer roofline of the
// hashing, measured on the GPU at hand): (bucket, sign) of n_keys synthetic keys for each
// of n_pairs (edge, row) parameter sets, with no memory traffic and no counter updates.
// The results are folded into one checksum so that no evaluation can be skipped.
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.cuh"

namespace cmpk {

namespace {

constexpr int kMbThreads = 512;
constexpr int kMbMaxPairs = 64;

// form 0: the key's powers x, x^2, x^3 shared by every pair (aggregated and int32-slab
// paths); form 1: the Horner form per pair (packed-slab path).  Keys are 0 .. n_keys - 1
// (below 2^31: the small-key arithmetic, as for every key of a 32-bit domain).
template <int FORM>
__global__ void __launch_bounds__(kMbThreads) k_cw_microbench(const cmp_hash* hash, int32_t n_pairs, int64_t n_keys,
                                                             uint32_t w_mask, uint32_t m31, uint32_t m4,
                                                             unsigned long long* out) {
  __shared__ PairParam prm[kMbMaxPairs];
  for (int p = threadIdx.x; p < n_pairs; p += blockDim.x) prm[p] = make_pair_param(hash[p]);
  __syncthreads();
  uint32_t acc = 0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n_keys; k += stride) {
    const uint64_t x = uint64_t(k);
    if (FORM == 0) {
      const KeyPow kp = key_powers(x);
      for (int p = 0; p < n_pairs; p++)
        acc += cw_bucket<true, true>(prm[p], kp, w_mask + 1) ^ uint32_t(cw_sign<true>(prm[p], kp));
    } else {
      const KeyX kx = key_x(x);
      for (int p = 0; p < n_pairs; p++) {
        const PairParam q = prm[p];
        const uint64_t c2 = q.c2_lo | (uint64_t(q.c2_hi) << 31), c1 = q.c1_lo | (uint64_t(q.c1_hi) << 31);
        acc += cw_bucket_h<true, true>(q, kx, w_mask + 1, m31, m4) ^ uint32_t(cw_sign_h<true>(q, kx, c2, c1, m31, m4));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicXor(out, (unsigned long long)acc);
}

}  // namespace

}  // namespace cmpk

using namespace cmpk;

extern "C" cmp_status cmp_microbench_cw(const cmp_hash* hash_dev, int32_t n_pairs, int64_t n_keys, int32_t w,
                                        int32_t form, uint64_t* out_dev, void* stream) {
  if (!hash_dev || !out_dev || n_pairs < 1 || n_pairs > kMbMaxPairs || n_keys < 0 || n_keys > (int64_t(1) << 31) ||
      w < 1 || (w & (w - 1)) || (form != 0 && form != 1))
    return CMP_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const unsigned grid = unsigned(sm_count()) * 4;
  if (form == 0)
    k_cw_microbench<0><<<grid, kMbThreads, 0, st>>>(hash_dev, n_pairs, n_keys, uint32_t(w - 1), 1u << 31, 4u,
                                                   reinterpret_cast<unsigned long long*>(out_dev));
  else
    k_cw_microbench<1><<<grid, kMbThreads, 0, st>>>(hash_dev, n_pairs, n_keys, uint32_t(w - 1), 1u << 31, 4u,
                                                   reinterpret_cast<unsigned long long*>(out_dev));
  return cudaGetLastError() == cudaSuccess ? CMP_OK : CMP_ECUDA;
}
