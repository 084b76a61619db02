// Learned estimate combiner (not in the paper, which takes the median over the d row
// estimates, Sec. 3.2): features from the exact row estimates and the sketches' self-join
// sizes, a 2-layer perceptron y = base + W2 relu(W1 x + b1) + b2 (base = max(x[skip], 0),
// a skip connection from the median row feature) with bfloat16 weights and fp32
// accumulation, and its training step (forward, backward, Adam) on the GPU.
//
// Parameters (fp32 master copy): W1[nh][nin], b1[nh], W2[nh], b2[1].  Every forward and
// backward pass uses their bfloat16 (nearest-even) roundings.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "estimate.cuh"

namespace cmpk {

constexpr int kMlpMaxIn = 66;      // d <= 64 row features + 2 self-join features
constexpr int kMlpMaxHidden = 64;
constexpr int kTrainSamples = 128;  // samples per CTA in the training kernel
constexpr float kFeatScale = 1.0f / 32.0f;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Thread-block cluster helpers: this CTA's rank in its cluster, a barrier of every thread of
// the cluster (release / acquire: shared-memory writes before it are visible after it), and
// the address of a shared variable in another CTA of the cluster.
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
template <class T>
__device__ __forceinline__ T* cluster_map_shared(T* p, unsigned rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
  return reinterpret_cast<T*>(out);
}

// ---------------------------------------------------------------- self-join sizes
// f2[s] = median over rows i of sum_j C[s][i][j]^2 (the Fast-AGMS self-join estimate of
// Sec. 3.2 applied to one sketch), exact per row, rounded once.  One cluster of kF2Cluster
// CTAs per sketch: CTA r of the cluster takes rows r, r + kF2Cluster, ..., its warps split
// each of them into contiguous parts, each lane streaming its part with four independent
// accumulators; after a cluster barrier the first CTA reads every row's exact sum from the
// other CTAs' shared memory (distributed shared memory) and takes the median.
constexpr int kF2Threads = 1024;
constexpr int kF2Cluster = 8;

__global__ void __launch_bounds__(kF2Threads) k_sketch_f2(const int32_t* __restrict__ C, int64_t n_sketches,
                                                          int32_t d, int32_t w, double* __restrict__ f2) {
  __shared__ u128 part[32];
  __shared__ i128 rows[CMP_MAX_D];  // this CTA's rows (the others: unused)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned rank = cluster_ctarank();
  const int64_t s = int64_t(blockIdx.x) / kF2Cluster;
  const int my_rows = (d - int(rank) + kF2Cluster - 1) / kF2Cluster;  // rows rank, rank + kF2Cluster, ...
  if (my_rows > 0) {
    const int split = nw / my_rows > 0 ? nw / my_rows : 1;
    const int units = my_rows * split;
    const int64_t len = (int64_t(w) + split - 1) / split;
    for (int u0 = 0; u0 < units; u0 += nw) {  // rounds of at most nw parts
      const int u = u0 + warp;
      if (u < units) {
        const int i = int(rank) + (u / split) * kF2Cluster, p = u % split;
        const int64_t b = int64_t(p) * len, e = b + len < w ? b + len : int64_t(w);
        const int32_t* src = C + (s * d + i) * int64_t(w);
        u128 a0 = 0, a1 = 0, a2 = 0, a3 = 0;  // each term < 2^62
        int64_t j = b + lane;
        for (; j + 96 < e; j += 128) {
          const int64_t v0 = __ldg(src + j), v1 = __ldg(src + j + 32), v2 = __ldg(src + j + 64),
                        v3 = __ldg(src + j + 96);
          a0 += u128(uint64_t(v0 * v0));
          a1 += u128(uint64_t(v1 * v1));
          a2 += u128(uint64_t(v2 * v2));
          a3 += u128(uint64_t(v3 * v3));
        }
        for (; j < e; j += 32) {
          const int64_t v = __ldg(src + j);
          a0 += u128(uint64_t(v * v));
        }
        u128 acc = a0 + a1 + a2 + a3;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const uint64_t lo = __shfl_down_sync(0xffffffffu, uint64_t(acc), off);
          const uint64_t hi = __shfl_down_sync(0xffffffffu, uint64_t(acc >> 64), off);
          acc += (u128(hi) << 64) | lo;
        }
        if (lane == 0) part[warp] = acc;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int q = 0; q < nw && u0 + q < units; q++) {
          const int uu = u0 + q, i = int(rank) + (uu / split) * kF2Cluster;
          if (uu % split == 0) rows[i] = 0;
          rows[i] = i128(u128(rows[i]) + part[q]);
        }
      }
      __syncthreads();
    }
  }
  cluster_sync_all();  // every row sum of the sketch is in its CTA's shared memory
  if (rank == 0 && threadIdx.x == 0) {
    i128 all[CMP_MAX_D];
    for (int i = 0; i < d; i++) all[i] = *cluster_map_shared(&rows[i], unsigned(i % kF2Cluster));
    for (int i = 1; i < d; i++) {  // insertion sort of exact integers
      const i128 v = all[i];
      int j = i - 1;
      while (j >= 0 && all[j] > v) {
        all[j + 1] = all[j];
        j--;
      }
      all[j + 1] = v;
    }
    const double r = (d & 1) ? i128_to_double(all[d / 2])
                             : 0.5 * mag_to_double(false, 0, u128(all[d / 2 - 1]) + u128(all[d / 2]));
    f2[s] = r;
  }
  cluster_sync_all();  // the other CTAs' shared memory stays until the first has read it
}

// ---------------------------------------------------------------- features
// v = sorted_i sign(E_i) ln(1 + |E_i|) / 32, m = d / 2 (the median slot):
// feat[q] = ( v_0 - v_m, ..., v_m, ..., v_{d-1} - v_m,  ln(1 + f2a[q]) / 32,  ln(1 + f2b[q]) / 32 )
// Centring the order statistics on the median keeps the inputs of a correction to the
// median small, so bfloat16 weights do not swamp it with rounding noise.
// f2a / f2b per sample, or (f2_idx != nullptr) both read from one per-sketch f2 array at
// f2_idx[2q], f2_idx[2q + 1] (-1: no sketch, feature of 0).
__global__ void k_mlp_features(const int64_t* __restrict__ row_est, int64_t n, int32_t d,
                               const double* __restrict__ f2a, const double* __restrict__ f2b,
                               const int32_t* __restrict__ f2_idx, float* __restrict__ feat) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float v[CMP_MAX_D];
  for (int i = 0; i < d; i++) {
    const u128 lo = uint64_t(row_est[(q * d + i) * 2]);
    const u128 hi = uint64_t(row_est[(q * d + i) * 2 + 1]);
    const double e = i128_to_double(i128((hi << 64) | lo));
    v[i] = float(copysign(log1p(fabs(e)), e)) * kFeatScale;
  }
  for (int i = 1; i < d; i++) {
    const float x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) {
      v[j + 1] = v[j];
      j--;
    }
    v[j + 1] = x;
  }
  float* out = feat + q * (d + 2);
  const float vm = v[d / 2];
  for (int i = 0; i < d; i++) out[i] = i == d / 2 ? vm : v[i] - vm;
  double fa, fb;
  if (f2_idx) {
    const int32_t ia = f2_idx[2 * q], ib = f2_idx[2 * q + 1];
    fa = ia >= 0 ? f2a[ia] : 0.0;
    fb = ib >= 0 ? f2a[ib] : 0.0;
  } else {
    fa = f2a[q];
    fb = f2b[q];
  }
  out[d] = float(log1p(fmax(fa, 0.0))) * kFeatScale;
  out[d + 1] = float(log1p(fmax(fb, 0.0))) * kFeatScale;
}

// ---------------------------------------------------------------- inference
__global__ void k_mlp_infer(const float* __restrict__ P, int32_t nin, int32_t nh, int32_t skip,
                            const float* __restrict__ x, int64_t n, float* __restrict__ y) {
  __shared__ float W[kMlpMaxHidden * kMlpMaxIn + 2 * kMlpMaxHidden + 1];
  const int np = nh * nin + 2 * nh + 1;
  for (int k = threadIdx.x; k < np; k += blockDim.x) W[k] = bf16r(P[k]);
  __syncthreads();
  const float* W1 = W;
  const float* b1 = W1 + nh * nin;
  const float* W2 = b1 + nh;
  const float b2 = W2[nh];
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
    float xs[kMlpMaxIn];
    for (int c = 0; c < nin; c++) xs[c] = x[s * nin + c];
    float acc = b2 + (skip >= 0 ? fmaxf(xs[skip], 0.f) : 0.f);
    for (int h = 0; h < nh; h++) {
      float z = b1[h];
      for (int c = 0; c < nin; c++) z = fmaf(W1[h * nin + c], xs[c], z);
      if (z > 0.f) acc = fmaf(W2[h], z, acc);
    }
    y[s] = acc;
  }
}

// ---------------------------------------------------------------- training
// Phase 1 (thread = sample): forward pass, d(loss)/dy = 2 (y - t) / n, activations and
// hidden gradients in shared memory.  Phase 2 (thread = parameter): this CTA's gradient
// contribution summed over its samples in a fixed order -> partial[cta][k].
__global__ void __launch_bounds__(kTrainSamples) k_mlp_grad(const float* __restrict__ P, int32_t nin, int32_t nh,
                                                           int32_t skip, const float* __restrict__ x,
                                                           const float* __restrict__ t,
                                                           int64_t n, float huber_delta, float* __restrict__ partial,
                                                           float* __restrict__ partial_loss) {
  // dynamic shared memory: W[np] | xs[S][nin] | act[S][nh] | dz[S][nh] | dys[S] | err2[S]
  extern __shared__ float shm[];
  const int np = nh * nin + 2 * nh + 1;
  float* W = shm;
  float* xsb = W + np;
  float* actb = xsb + kTrainSamples * nin;
  float* dzb = actb + kTrainSamples * nh;
  float* dys = dzb + kTrainSamples * nh;
  float* err2 = dys + kTrainSamples;
  auto xs = [&](int s, int c) -> float& { return xsb[s * nin + c]; };
  auto act = [&](int s, int h) -> float& { return actb[s * nh + h]; };
  auto dz = [&](int s, int h) -> float& { return dzb[s * nh + h]; };
  for (int k = threadIdx.x; k < np; k += blockDim.x) W[k] = bf16r(P[k]);
  __syncthreads();
  const float* W1 = W;
  const float* b1 = W1 + nh * nin;
  const float* W2 = b1 + nh;
  const float b2 = W2[nh];
  const int64_t s0 = int64_t(blockIdx.x) * kTrainSamples;
  const int ns = int(min(int64_t(kTrainSamples), n - s0));
  const int si = threadIdx.x;
  if (si < ns) {
    const int64_t s = s0 + si;
    for (int c = 0; c < nin; c++) xs(si, c) = x[s * nin + c];
    float acc = b2 + (skip >= 0 ? fmaxf(xs(si, skip), 0.f) : 0.f);
    for (int h = 0; h < nh; h++) {
      float z = b1[h];
      for (int c = 0; c < nin; c++) z = fmaf(W1[h * nin + c], xs(si, c), z);
      act(si, h) = z > 0.f ? z : 0.f;
      if (z > 0.f) acc = fmaf(W2[h], z, acc);
    }
    const float e = acc - t[s];
    float dy;
    if (huber_delta > 0.f) {  // Huber: quadratic within delta, linear beyond
      const float a = fabsf(e);
      dy = (a <= huber_delta ? e : copysignf(huber_delta, e)) / float(n);
      err2[si] = a <= huber_delta ? 0.5f * e * e : huber_delta * (a - 0.5f * huber_delta);
    } else {
      dy = 2.f * e / float(n);
      err2[si] = e * e;
    }
    dys[si] = dy;
    for (int h = 0; h < nh; h++) dz(si, h) = act(si, h) > 0.f ? dy * W2[h] : 0.f;
  }
  __syncthreads();
  float* out = partial + int64_t(blockIdx.x) * np;
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    float g = 0.f;
    if (k < nh * nin) {
      const int h = k / nin, c = k % nin;
      for (int s = 0; s < ns; s++) g = fmaf(dz(s, h), xs(s, c), g);
    } else if (k < nh * nin + nh) {
      const int h = k - nh * nin;
      for (int s = 0; s < ns; s++) g += dz(s, h);
    } else if (k < nh * nin + 2 * nh) {
      const int h = k - nh * nin - nh;
      for (int s = 0; s < ns; s++) g = fmaf(dys[s], act(s, h), g);
    } else {
      for (int s = 0; s < ns; s++) g += dys[s];
    }
    out[k] = g;
  }
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int s = 0; s < ns; s++) l += err2[s];
    partial_loss[blockIdx.x] = l;
  }
}

// Sum of the CTA partials in a fixed order, then one Adam step (Kingma & Ba 2015) on the
// fp32 master parameters.
__global__ void k_mlp_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v, int32_t np,
                           const float* __restrict__ partial, const float* __restrict__ partial_loss, int32_t n_cta,
                           int64_t n, float lr, int32_t step, float* __restrict__ loss, float* __restrict__ grad) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, float(step)), c2 = 1.f - powf(b2, float(step));
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    float g = 0.f;
    for (int c = 0; c < n_cta; c++) g += partial[int64_t(c) * np + k];
    if (grad) grad[k] = g;
    const float mk = b1 * m[k] + (1.f - b1) * g;
    const float vk = b2 * v[k] + (1.f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    P[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
    float l = 0.f;
    for (int c = 0; c < n_cta; c++) l += partial_loss[c];
    *loss = l / float(n);
  }
}

// Combined estimate: the plain median where it is a usable join size (>= 1 tuple), the
// network's prediction exp(32 y) - 1 where the median is below one tuple.
__global__ void k_mlp_combine(const double* __restrict__ median, const float* __restrict__ y,
                              const uint8_t* __restrict__ eligible, int64_t n, double use_median_at,
                              double* __restrict__ out) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double m = median[q];
  const bool net = (!eligible || eligible[q]) && !(m >= use_median_at);
  out[q] = net ? fmax(expm1(32.0 * double(y[q])), 0.0) : m;
}

cudaError_t launch_sketch_f2(const int32_t* C, int64_t n_sketches, int32_t d, int32_t w, double* f2,
                             cudaStream_t st) {
  if (n_sketches <= 0) return cudaSuccess;
  if (n_sketches > (int64_t(1) << 31) / kF2Cluster - 1) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(n_sketches * kF2Cluster));  // one cluster per sketch
  cfg.blockDim = dim3(unsigned(kF2Threads));
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kF2Cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_sketch_f2, C, n_sketches, d, w, f2);
}

cudaError_t launch_mlp_features(const int64_t* row_est, int64_t n, int32_t d, const double* f2a, const double* f2b,
                                float* feat, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_mlp_features<<<unsigned((n + 127) / 128), 128, 0, st>>>(row_est, n, d, f2a, f2b, nullptr, feat);
  return cudaGetLastError();
}

cudaError_t launch_mlp_features_indexed(const int64_t* row_est, int64_t n, int32_t d, const double* f2,
                                        const int32_t* f2_idx, float* feat, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_mlp_features<<<unsigned((n + 127) / 128), 128, 0, st>>>(row_est, n, d, f2, nullptr, f2_idx, feat);
  return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const float* P, int32_t nin, int32_t nh, int32_t skip, const float* x, int64_t n,
                             float* y, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_mlp_infer<<<unsigned(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(P, nin, nh, skip, x, n, y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_combine(const double* median, const float* y, int64_t n, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_mlp_combine<<<unsigned((n + 255) / 256), 256, 0, st>>>(median, y, nullptr, n, 1.0, out);
  return cudaGetLastError();
}

int64_t mlp_train_ctas(int64_t n) { return (n + kTrainSamples - 1) / kTrainSamples; }

cudaError_t launch_mlp_train(float* P, float* m, float* v, int32_t nin, int32_t nh, int32_t skip, const float* x,
                             const float* t, int64_t n, float huber_delta, float lr, int32_t step, float* loss,
                             float* grad, float* partial,
                             float* partial_loss, cudaStream_t st) {
  const int64_t ctas = mlp_train_ctas(n);
  const int32_t np = nh * nin + 2 * nh + 1;
  if (ctas > 0) {
    const size_t smem = sizeof(float) * size_t(np + kTrainSamples * (nin + 2 * nh + 2));
    cudaError_t e0 = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e0 != cudaSuccess) return e0;
    k_mlp_grad<<<unsigned(ctas), kTrainSamples, smem, st>>>(P, nin, nh, skip, x, t, n, huber_delta, partial,
                                                            partial_loss);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_mlp_adam<<<unsigned((np + 255) / 256), 256, 0, st>>>(P, m, v, np, partial, partial_loss, int32_t(ctas), n, lr,
                                                         step, loss, grad);
  return cudaGetLastError();
}

}  // namespace cmpk

using namespace cmpk;

extern "C" {

int64_t cmp_mlp_param_count(int32_t nin, int32_t nh) {
  if (nin < 1 || nin > kMlpMaxIn || nh < 1 || nh > kMlpMaxHidden) return -1;
  return int64_t(nh) * nin + 2 * nh + 1;
}

cmp_status cmp_sketch_f2(const int32_t* counters_dev, int64_t n_sketches, int32_t d, int32_t w, double* f2_dev,
                         void* stream) {
  if (n_sketches < 0 || d < 1 || d > CMP_MAX_D || w < 1 || w > CMP_MAX_W) return CMP_EINVAL;
  if (n_sketches > 0 && (!counters_dev || !f2_dev)) return CMP_EINVAL;
  return launch_sketch_f2(counters_dev, n_sketches, d, w, f2_dev, reinterpret_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

cmp_status cmp_mlp_features(const int64_t* row_est_dev, int64_t n, int32_t d, const double* f2a_dev,
                            const double* f2b_dev, float* feat_dev, void* stream) {
  if (n < 0 || d < 1 || d > CMP_MAX_D) return CMP_EINVAL;
  if (n > 0 && (!row_est_dev || !f2a_dev || !f2b_dev || !feat_dev)) return CMP_EINVAL;
  return launch_mlp_features(row_est_dev, n, d, f2a_dev, f2b_dev, feat_dev, reinterpret_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

cmp_status cmp_mlp_features_indexed(const int64_t* row_est_dev, int64_t n, int32_t d, const double* f2_dev,
                                    const int32_t* f2_index_dev, float* feat_dev, void* stream) {
  if (n < 0 || d < 1 || d > CMP_MAX_D) return CMP_EINVAL;
  if (n > 0 && (!row_est_dev || !f2_dev || !f2_index_dev || !feat_dev)) return CMP_EINVAL;
  return launch_mlp_features_indexed(row_est_dev, n, d, f2_dev, f2_index_dev, feat_dev,
                                     reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

cmp_status cmp_mlp_infer(const float* params_dev, int32_t nin, int32_t nh, int32_t skip, const float* x_dev, int64_t n,
                         float* y_dev, void* stream) {
  if (cmp_mlp_param_count(nin, nh) < 0 || n < 0 || skip < -1 || skip >= nin) return CMP_EINVAL;
  if (!params_dev || (n > 0 && (!x_dev || !y_dev))) return CMP_EINVAL;
  return launch_mlp_infer(params_dev, nin, nh, skip, x_dev, n, y_dev, reinterpret_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

cmp_status cmp_mlp_combine_ex(const double* median_dev, const float* y_dev, const uint8_t* eligible_dev, int64_t n,
                              double use_median_at, double* est_dev, void* stream) {
  if (n < 0 || (n > 0 && (!median_dev || !y_dev || !est_dev)) || use_median_at != use_median_at) return CMP_EINVAL;
  if (n == 0) return CMP_OK;
  k_mlp_combine<<<unsigned((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      median_dev, y_dev, eligible_dev, n, use_median_at, est_dev);
  return cudaGetLastError() == cudaSuccess ? CMP_OK : CMP_ECUDA;
}

cmp_status cmp_mlp_combine(const double* median_dev, const float* y_dev, int64_t n, double* est_dev, void* stream) {
  if (n < 0 || (n > 0 && (!median_dev || !y_dev || !est_dev))) return CMP_EINVAL;
  return launch_mlp_combine(median_dev, y_dev, n, est_dev, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

size_t cmp_mlp_train_ws_bytes(int32_t nin, int32_t nh, int64_t n) {
  const int64_t np = cmp_mlp_param_count(nin, nh);
  if (np < 0 || n < 0) return 0;
  const int64_t ctas = mlp_train_ctas(n);
  return size_t(align16(sizeof(float) * size_t(ctas * np)) + align16(sizeof(float) * size_t(ctas > 0 ? ctas : 1)));
}

cmp_status cmp_mlp_train_step(float* params_dev, float* adam_m_dev, float* adam_v_dev, int32_t nin, int32_t nh,
                              int32_t skip, const float* x_dev, const float* y_dev, int64_t n, float huber_delta,
                              float lr, int32_t step, float* loss_dev, float* grad_dev, void* ws_dev, size_t ws_bytes,
                              void* stream) {
  const int64_t np = cmp_mlp_param_count(nin, nh);
  if (np < 0 || n < 1 || step < 1 || !(lr > 0.f) || skip < -1 || skip >= nin || !(huber_delta >= 0.f))
    return CMP_EINVAL;
  if (!params_dev || !adam_m_dev || !adam_v_dev || !x_dev || !y_dev) return CMP_EINVAL;
  if (ws_bytes < cmp_mlp_train_ws_bytes(nin, nh, n) || !ws_dev) return CMP_EWORKSPACE;
  const int64_t ctas = mlp_train_ctas(n);
  float* partial = static_cast<float*>(ws_dev);
  float* partial_loss =
      reinterpret_cast<float*>(static_cast<unsigned char*>(ws_dev) + align16(sizeof(float) * size_t(ctas * np)));
  return launch_mlp_train(params_dev, adam_m_dev, adam_v_dev, nin, nh, skip, x_dev, y_dev, n, huber_delta, lr, step,
                          loss_dev, grad_dev,
                          partial, partial_loss, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? CMP_OK
             : CMP_ECUDA;
}

}  // extern "C"
