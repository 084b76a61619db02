// cmp_estimate_noalloc: the sub-plan estimate with its workspace in a fixed array of the
// library's own device memory instead of a caller-provided buffer, for callers that may
// not allocate device memory themselves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "estimate.cuh"

using namespace cmpk;

namespace {

// The workspace: CMP_NOALLOC_WS_BYTES bytes that every GPU loading the library holds
// until the process exits.  Host code must not take this name as a device address; it
// uses the address cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_ws[CMP_NOALLOC_WS_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the workspace.
cmp_status workspace_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CMP_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || !p) return CMP_ECUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CMP_OK;
}

}  // namespace

extern "C" cmp_status cmp_estimate_noalloc(const void* plan_host, const void* plan_dev, double* est_dev,
                                           int64_t* row_est_dev, int32_t* status_dev, void* stream) {
  if (!plan_host || !plan_dev) return CMP_EINVAL;
  EstPlanHdr H;
  std::memcpy(&H, plan_host, sizeof(H));
  if (H.magic != kEstPlanMagic || H.version != kEstPlanVersion) return CMP_EINVAL;
  if (H.n_sub > 0 && !est_dev) return CMP_EINVAL;
  // Layout (est_args): per-item partial sums and caches, then `grid` generic per-CTA
  // scratch areas, then `slots` triangle rows.  est_args places the triangle rows after
  // grid >= 1 CTA areas whether or not the plan has generic items, so one CTA area is
  // always reserved; triangle rows beyond what fits run in successive waves.
  const size_t cap = size_t(CMP_NOALLOC_WS_BYTES), fixed = est_fixed_bytes(H);
  const size_t per_cta = size_t(H.scratch_per_cta);
  const size_t per_tri = H.n_tri > 0 ? size_t(H.tri_row_bytes) : 0;
  if (fixed + per_cta + per_tri > cap) return CMP_EWORKSPACE;
  int64_t grid = std::max<int64_t>(1, H.grid);
  if (per_cta) grid = std::max<int64_t>(1, std::min<int64_t>(grid, int64_t((cap - fixed - per_tri) / per_cta)));
  int64_t slots = 0;
  if (per_tri) slots = std::min<int64_t>(H.n_tri * H.d, int64_t((cap - fixed - per_cta * size_t(grid)) / per_tri));
  // the exact tier's kernel reuses the scratch region: as many of its CTA areas as fit (at least one)
  int64_t wide_ctas = 1;
  if (H.wide && H.wide_scratch_per_cta > 0 && cap > fixed)
    wide_ctas = std::max<int64_t>(1, std::min<int64_t>(H.wide_grid, int64_t((cap - fixed) / size_t(H.wide_scratch_per_cta))));
  if (est_ws_bytes(H, grid, slots, wide_ctas) > cap || (per_tri && slots < 1)) return CMP_EWORKSPACE;
  void* ws_v = nullptr;
  const cmp_status st = workspace_address(&ws_v);
  if (st != CMP_OK) return st;
  const EstArgs a = est_args(H, static_cast<const unsigned char*>(plan_dev), static_cast<unsigned char*>(ws_v),
                             int32_t(grid), slots, status_dev, int32_t(wide_ctas));
  return launch_estimate(a, H, est_dev, row_est_dev, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? CMP_OK
                                                                                                          : CMP_ECUDA;
}
