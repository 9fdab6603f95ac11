// Allocation-free forward render: gs_render_fwd_noalloc.
//
// Some callers of this library cannot call cudaMalloc: code that runs inside
// a host framework that owns all device memory (an inference-engine plugin, a
// middleware node handed fixed buffers), or a real-time loop where
// cudaMalloc's implicit device synchronisation is not acceptable.  This entry
// point renders with the same kernels as gs_project + gs_bin_sort +
// gs_render_fwd, but its workspace is a file-scope device array of fixed size
// (GS_NOALLOC_SCRATCH_BYTES) instead of a caller buffer; the caller still
// passes every input and output.
#include <mutex>

#include "gs_internal.h"

namespace gsb {

// The scratch workspace.  In host code this name is only a stand-in: the
// device address is fetched once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device; the first call
// per device looks it up (with that device current) and caches it.
static gs_status noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return GS_OK;
}

__global__ void k_noalloc_status(const uint32_t* counters, int32_t* status_dev) {
  *status_dev = (int32_t)counters[kStatus];
}

}  // namespace gsb

using namespace gsb;

extern "C" gs_status gs_render_fwd_noalloc(const gs_map* map, const gs_camera* cams_dev, const gs_frame* frame,
                                           const gs_config* cfg, float* rgb, float* depth, float* opac,
                                           float* t_final, uint32_t* n_contrib, int32_t* status_dev,
                                           gs_stream_t stream) {
  if (!map || !cams_dev || !frame || !cfg || !t_final || !n_contrib || !status_dev) return GS_ERR_ARG;
  if (map->n < 1 || map->sh_degree < 0 || map->sh_degree > 3 || (map->sh_bf16 != 0 && map->sh_bf16 != 1) ||
      !map->mean || !map->log_scale || !map->quat || !map->logit_opacity || !map->sh_dc ||
      (map->sh_degree > 0 && !map->sh_rest))
    return GS_ERR_ARG;
  if (!(cfg->alpha_min > 0.f && cfg->alpha_min < 1.f) || !(cfg->alpha_max >= cfg->alpha_min && cfg->alpha_max < 1.f) ||
      !(cfg->t_min > 0.f && cfg->t_min < 1.f) || !(cfg->near_z > 0.f) || !(cfg->dilation >= 0.f) ||
      !(cfg->fov_clamp > 0.f))
    return GS_ERR_ARG;
  // Size the pair buffer from what the fixed array leaves over; reject
  // requests whose per-Gaussian and per-tile parts alone do not fit.
  gs_layout L;
  if (gs_workspace_layout(map->n, frame, 1, &L) != GS_OK) return GS_ERR_ARG;
  const size_t limit = (size_t)GS_NOALLOC_SCRATCH_BYTES;
  if (L.total > limit) return GS_ERR_UNSUPPORTED;
  // largest pair capacity whose layout fits (the layout grows with it)
  int64_t lo = 1, hi = (int64_t)(limit - L.total);
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo + 1) / 2;
    if (gs_workspace_layout(map->n, frame, mid, &L) == GS_OK && L.total <= limit) lo = mid;
    else hi = mid - 1;
  }
  const int64_t cap = lo;
  if (gs_workspace_layout(map->n, frame, cap, &L) != GS_OK || L.total > limit) return GS_ERR_UNSUPPORTED;
  void* base = nullptr;
  gs_status s = noalloc_scratch(&base);
  if (s != GS_OK) return s;
  gs_workspace ws;
  ws.ptr = base;
  ws.n = map->n;
  ws.pair_capacity = cap;
  ws.frame = *frame;
  const Ws w = resolve_ws(&ws, L);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // launch_project clears the counters and the per-tile counts that the
  // later kernels start from; every other part is written before it is read.
  if (launch_project(*map, cams_dev, *cfg, w, st) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_bin_sort(w, st) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_render_fwd(*cfg, w, rgb, depth, opac, t_final, n_contrib, st) != cudaSuccess) return GS_ERR_CUDA;
  k_noalloc_status<<<1, 1, 0, st>>>(w.counters, status_dev);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
