// Test support (no counterpart in the paper): one pass of the library's
// stable radix sort over a small synthetic array, to show that its only
// device wait - a tile's bounded look-back on the tiles before it - ends on
// its own.  With skip_first_tile set, the pass's ticket counter starts at 1,
// so no CTA ever takes tile 0 and the wait of tile 1 on tile 0 runs out:
// after kSpinLimit polls the sort's error word becomes GS_ERR_TIMEOUT and
// the pass still writes only in-range slots.  Without it the pass is an
// ordinary stable sort by the low 8 bits of the keys.
#include "gs_internal.h"
#include "radix.cuh"

namespace gsb {

constexpr int kProbeTiles = 2;
constexpr int kProbeItems = kProbeTiles * kRadixTileEntries;
// scratch words: [0] error word, [1] item count, [2..8) tickets, [64..) digit
// counts [6][256], then tile status words [6][kProbeTiles][256], then keys in,
// entries in, keys out, entries out (kProbeItems each)
constexpr size_t kProbeCounts = 64;
constexpr size_t kProbeTileWords = kProbeCounts + 6 * 256;
constexpr size_t kProbeKeys = kProbeTileWords + 6 * kProbeTiles * 256;
constexpr size_t kProbeWords = kProbeKeys + 4 * (size_t)kProbeItems;

struct LowByteDigit {
  __device__ __forceinline__ uint32_t operator()(uint32_t key, uint32_t, int) const { return key & 255u; }
};

// One CTA: clears the scratch, writes keys k(i) = (i * 2654435761) >> 24 and
// entries i, their digit counts, and the first ticket.
__global__ void __launch_bounds__(256) k_probe_init(uint32_t* s, uint32_t first_ticket) {
  for (size_t i = threadIdx.x; i < kProbeKeys; i += blockDim.x) s[i] = 0;
  __syncthreads();
  uint32_t* key = s + kProbeKeys;
  uint32_t* val = key + kProbeItems;
  for (int i = threadIdx.x; i < kProbeItems; i += blockDim.x) {
    const uint32_t k = ((uint32_t)i * 2654435761u) >> 24;
    key[i] = k;
    val[i] = (uint32_t)i;
    atomicAdd(s + kProbeCounts + (k & 255u), 1u);  // pass 0's digit counts
  }
  if (threadIdx.x == 0) {
    s[1] = kProbeItems;
    s[2] = first_ticket;
  }
}

__global__ void k_probe_status(const uint32_t* s, int32_t* out) { *out = (int32_t)s[0]; }

}  // namespace gsb

using namespace gsb;

extern "C" size_t gs_sort_wait_probe_bytes(void) { return kProbeWords * sizeof(uint32_t); }

extern "C" gs_status gs_sort_wait_probe(void* scratch_dev, size_t scratch_bytes, int32_t skip_first_tile,
                                        int32_t* status_dev, gs_stream_t stream) {
  if (!scratch_dev || !status_dev || scratch_bytes < kProbeWords * sizeof(uint32_t)) return GS_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(scratch_dev) & 15) != 0) return GS_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* s = static_cast<uint32_t*>(scratch_dev);
  k_probe_init<<<1, 256, 0, st>>>(s, skip_first_tile ? 1u : 0u);
  RadixScratch rs;
  rs.n = s + 1;
  rs.status = s;
  rs.counts = s + kProbeCounts;
  rs.tiles = s + kProbeTileWords;
  rs.tickets = s + 2;
  rs.tiles_max = kProbeTiles;
  uint32_t* key = s + kProbeKeys;
  uint32_t* val = key + kProbeItems;
  k_radix_pass<<<1, kRadixThreads, 0, st>>>(rs, LowByteDigit{}, 0, key, val, val + kProbeItems,
                                            val + 2 * kProbeItems);
  k_probe_status<<<1, 1, 0, st>>>(s, status_dev);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
