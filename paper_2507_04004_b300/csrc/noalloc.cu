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
// device address is fetched once per device (and again after the device's
// context changed) with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
// Per device: the scratch address and the id of the CUDA context it was
// looked up in.  A device reset (cudaDeviceReset) or a new primary context
// loads the module again, possibly at another address, so the address is
// looked up again whenever the current context's id differs from the cached one.
struct NoallocSlot {
  void* addr = nullptr;
  unsigned long long ctx_id = 0;
};
static NoallocSlot g_noalloc_slot[kMaxDevices];

// Id of the current CUDA context (cuCtxGetCurrent + cuCtxGetId, reached
// through the runtime's driver entry-point query so that the library needs
// no link to the driver library); false if it cannot be read.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
static bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {  // under g_noalloc_mu
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
        q0 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
      get_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
    resolved = true;
  }
  if (!get_current || !get_id) return false;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current device's context.  The
// first call per device (and the first after its context changed) looks it
// up with cudaGetSymbolAddress, with that device current, and caches it.  If
// the context id cannot be read, every call outside stream capture looks the
// address up again.
static gs_status noalloc_scratch(cudaStream_t st, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return GS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocSlot& slot = g_noalloc_slot[dev];
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  const bool fresh = slot.addr && (have_id ? slot.ctx_id == id : cap != cudaStreamCaptureStatusNone);
  if (!fresh) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
    // the symbol lookup made the device's primary context current if it was not
    if (!have_id) current_context_id(&id);
    slot.addr = p;
    slot.ctx_id = id;
  }
  *out = slot.addr;
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
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* base = nullptr;
  gs_status s = noalloc_scratch(st, &base);
  if (s != GS_OK) return s;
  gs_workspace ws;
  ws.ptr = base;
  ws.n = map->n;
  ws.pair_capacity = cap;
  ws.frame = *frame;
  const Ws w = resolve_ws(&ws, L);
  // launch_project clears the counters and the per-tile counts that the
  // later kernels start from; every other part is written before it is read.
  if (launch_project(*map, cams_dev, *cfg, w, st) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_bin_sort(w, st) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_render_fwd(*cfg, w, rgb, depth, opac, t_final, n_contrib, st) != cudaSuccess) return GS_ERR_CUDA;
  k_noalloc_status<<<1, 1, 0, st>>>(w.counters, status_dev);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
