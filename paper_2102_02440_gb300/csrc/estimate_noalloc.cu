// cmp_estimate_noalloc: the sub-plan estimate with its workspace in a fixed array of the
// library's own device memory instead of a caller-provided buffer, for callers that may
// not allocate device memory themselves.
#include <cuda_runtime.h>

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
  if (H.magic != kEstPlanMagic || H.version != 1) return CMP_EINVAL;
  if (H.n_sub > 0 && !est_dev) return CMP_EINVAL;
  // per-item partial sums, then as many per-CTA scratch areas as fit (at least one)
  const size_t fixed = align16(sizeof(i128) * size_t(H.n_items)) + align16(sizeof(int32_t) * size_t(H.n_items));
  const size_t per_cta = size_t(H.scratch_per_cta);
  if (fixed + per_cta > size_t(CMP_NOALLOC_WS_BYTES)) return CMP_EWORKSPACE;
  size_t fit = per_cta ? (size_t(CMP_NOALLOC_WS_BYTES) - fixed) / per_cta : size_t(H.grid);
  const int32_t grid = int32_t(fit < size_t(H.grid) ? fit : size_t(H.grid));
  void* ws_v = nullptr;
  const cmp_status st = workspace_address(&ws_v);
  if (st != CMP_OK) return st;
  unsigned char* ws = static_cast<unsigned char*>(ws_v);
  const unsigned char* pd = static_cast<const unsigned char*>(plan_dev);
  EstArgs a;
  std::memset(&a, 0, sizeof(a));
  a.subs = reinterpret_cast<const EstSub*>(pd + H.off_subs);
  a.ops = reinterpret_cast<const EstOp*>(pd + H.off_ops);
  a.inputs = reinterpret_cast<const EstIn*>(pd + H.off_in);
  a.items = reinterpret_cast<const EstItem*>(pd + H.off_items);
  a.partial = reinterpret_cast<i128*>(ws);
  a.partial_ovf = reinterpret_cast<int32_t*>(ws + align16(sizeof(i128) * size_t(H.n_items)));
  a.scratch = ws + fixed;
  a.scratch_per_cta = H.scratch_per_cta;
  a.n_items = H.n_items;
  a.n_sub = H.n_sub;
  a.d = H.d;
  a.w = H.w;
  a.max_slots = H.max_slots;
  a.max_in = H.max_in;
  a.max_suf = H.max_suf;
  a.max_rank = H.max_rank;
  a.grid = grid > 0 ? grid : 1;
  a.threads = H.threads;
  a.status = status_dev;
  return launch_estimate(a, est_dev, row_est_dev, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? CMP_OK
                                                                                                          : CMP_ECUDA;
}
