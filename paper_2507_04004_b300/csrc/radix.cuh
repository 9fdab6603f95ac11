// Stable LSD radix sort of (key, value) pairs of 32-bit words by 8-bit
// digits, "onesweep": the digit counts of every pass come from one read of
// the items (the counts do not depend on the order), and each pass is one
// kernel whose CTAs take tiles of kSortTile consecutive items by ticket, rank
// them stably, and find where their run of each digit starts by looking back
// over the earlier tiles' published counts (decoupled look-back).  A tile's
// status word per digit: bits 30-31 = 1 (its own count in bits 0-29) or 2
// (the count of all tiles up to and including it), so fewer than 2^30 items.
// Waits on an earlier tile are bounded: past kSpinLimit polls the sort's
// error word becomes GS_ERR_TIMEOUT and the pass writes only in-range slots.
// The digit of an item is a functor Digit(key, value, pass) < 256.
#pragma once

#include "gs_internal.h"

namespace gsb {

constexpr int kRadixThreads = 256;

__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Lanes of the warp whose (active) digit equals this lane's: the AND of the
// eight ballots of the digit's bits, each taken as is or complemented.
__device__ __forceinline__ unsigned digit_peers(uint32_t d, bool act) {
  unsigned peers = __ballot_sync(kFull, act);
#pragma unroll
  for (int bit = 0; bit < 8; ++bit) {
    const bool on = (d >> bit) & 1u;
    const unsigned m = __ballot_sync(kFull, on);
    peers &= on ? m : ~m;
  }
  return peers;
}

constexpr int kSortItems = 8;                            // items per thread
constexpr int kSortTile = kRadixThreads * kSortItems;    // items per tile
static_assert(kSortTile == kRadixTileEntries, "tile size of the sort");
constexpr uint32_t kFlagAgg = 1u << 30, kFlagPrefix = 2u << 30, kValueMask = (1u << 30) - 1u;
constexpr int kSpinLimit = 1 << 16;
constexpr int kLookBack = 16;  // earlier tiles' status words read per round trip

// Device pointers of one sort: the item count, the error word (the kernels
// do nothing while it is nonzero and set GS_ERR_TIMEOUT when a wait gives
// up), digit counts [6][256] (zero before k_radix_counts), per-tile status
// words [6][tiles_max][256], tile tickets [6] (zero before each pass).
struct RadixScratch {
  const uint32_t* n;
  uint32_t* status;
  uint32_t* counts;
  uint32_t* tiles;
  uint32_t* tickets;
  int64_t tiles_max;
};

// Digit counts of every pass over all items (added to the zeroed counts);
// clears the tile status words the passes will use.  Work of CTA `cta` of
// `ncta` CTAs of kRadixThreads threads.
template <class Digit>
__device__ __forceinline__ void radix_counts(const RadixScratch& rs, Digit dg, int passes,
                                             const uint32_t* __restrict__ key, const uint32_t* __restrict__ val,
                                             uint32_t cta, uint32_t ncta) {
  __shared__ uint32_t h[6][256];
  if (*rs.status != 0) return;
  const uint64_t n = *rs.n;
  const uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
  const uint64_t tid = (uint64_t)cta * kRadixThreads + threadIdx.x, stride = (uint64_t)ncta * kRadixThreads;
  for (int p = 0; p < passes; ++p) {
    uint32_t* st = rs.tiles + (int64_t)p * rs.tiles_max * 256;
    for (uint64_t i = tid; i < ntiles * 256; i += stride) st[i] = 0;
  }
  for (int i = threadIdx.x; i < 6 * 256; i += kRadixThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  for (uint64_t i = tid; i < n; i += stride) {
    const uint32_t k = key[i], v = val[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][dg(k, v, p)], 1u);
  }
  __syncthreads();
  uint32_t* g = rs.counts;
  for (int i = threadIdx.x; i < passes * 256; i += kRadixThreads) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(g + i, c);
  }
}

template <class Digit>
__global__ void __launch_bounds__(kRadixThreads) k_radix_counts(RadixScratch rs, Digit dg, int passes,
                                                                const uint32_t* __restrict__ key,
                                                                const uint32_t* __restrict__ val) {
  radix_counts(rs, dg, passes, key, val, blockIdx.x, gridDim.x);
}

// One LSD pass: stable scatter of the items by the pass's digit.
template <class Digit>
__global__ void __launch_bounds__(kRadixThreads) k_radix_pass(RadixScratch rs, Digit dg, int pass,
                                                              const uint32_t* __restrict__ key_in,
                                                              const uint32_t* __restrict__ val_in,
                                                              uint32_t* __restrict__ key_out,
                                                              uint32_t* __restrict__ val_out) {
  constexpr int NW = kRadixThreads / 32;
  __shared__ uint32_t s_wcnt[NW][256];  // per warp: count of each digit, then its first slot in the tile
  __shared__ uint32_t s_base[256];      // first output slot of each digit's run of this tile
  __shared__ uint32_t s_local[256];     // first slot of each digit's run inside the tile
  __shared__ uint32_t s_wsum[NW];
  __shared__ uint32_t s_key[kSortTile], s_val[kSortTile];  // the tile in digit order
  __shared__ uint32_t s_ticket;
  if (*rs.status != 0) return;
  const uint64_t n = *rs.n;
  const uint32_t ntiles = (uint32_t)((n + kSortTile - 1) / kSortTile);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt(lane);
  uint32_t* status = rs.tiles + (int64_t)pass * rs.tiles_max * 256;
  const uint32_t* counts = rs.counts + pass * 256;
  for (;;) {
    for (int i = threadIdx.x; i < NW * 256; i += kRadixThreads) (&s_wcnt[0][0])[i] = 0;
    if (threadIdx.x == 0) s_ticket = atomicAdd(rs.tickets + pass, 1u);
    __syncthreads();
    const uint32_t t = s_ticket;
    if (t >= ntiles) return;
    // this warp's 256 entries, taken lane-minor: entry order = (j, lane) order
    const uint64_t base = (uint64_t)t * kSortTile + (uint64_t)warp * 32 * kSortItems;
    uint32_t k[kSortItems], v[kSortItems], d[kSortItems], r[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const uint64_t i = base + 32 * j + lane;
      k[j] = i < n ? key_in[i] : 0u;
      v[j] = i < n ? val_in[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const bool act = base + 32 * j + lane < n;
      d[j] = dg(k[j], v[j], pass);
      const unsigned peers = digit_peers(d[j], act);
      const uint32_t prev = s_wcnt[warp][d[j]];
      r[j] = prev + __popc(peers & lt);
      __syncwarp();
      if (act && (peers & lt) == 0) s_wcnt[warp][d[j]] = prev + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      const int dd = threadIdx.x;
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = s_wcnt[w][dd];
        s_wcnt[w][dd] = run;
        run += c;
      }
      // publish this tile's count, then look back for the runs of earlier tiles
      volatile uint32_t* st = status;
      st[(int64_t)t * 256 + dd] = (t == 0 ? kFlagPrefix : kFlagAgg) | run;
      uint32_t excl = 0;
      if (t > 0) {
        // kLookBack earlier tiles' words are loaded per round trip, nearest first
        bool found = false;
        for (int64_t tt = (int64_t)t - 1; tt >= 0 && !found; tt -= kLookBack) {
          uint32_t w[kLookBack];
#pragma unroll
          for (int q = 0; q < kLookBack; ++q) w[q] = tt - q >= 0 ? (uint32_t)st[(tt - q) * 256 + dd] : (uint32_t)kFlagPrefix;
#pragma unroll
          for (int q = 0; q < kLookBack; ++q) {
            if (found) break;
            for (int spin = 0; (w[q] >> 30) == 0; ++spin) {  // that tile has not published yet
              if (spin >= kSpinLimit) {
                atomicExch(rs.status, (uint32_t)GS_ERR_TIMEOUT);
                w[q] = kFlagPrefix;
                break;
              }
              __nanosleep(64);
              w[q] = st[(tt - q) * 256 + dd];
            }
            excl += w[q] & kValueMask;
            found = (w[q] >> 30) == 2u;
          }
        }
        st[(int64_t)t * 256 + dd] = kFlagPrefix | (excl + run);
      }
      // first slot of the digit: all entries of lower digits, then earlier tiles
      s_base[dd] = excl;
      // the digit's first slot inside the tile: exclusive scan of the tile's counts
      const uint32_t inc = warp_incl_scan(run, lane);
      if (lane == 31) s_wsum[warp] = inc;
      s_local[dd] = inc - run;
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t add = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) add += w < warp ? s_wsum[w] : 0u;
      s_local[threadIdx.x] += add;
    }
    __syncthreads();
    // exclusive scan of the pass's digit counts (one warp), added to s_base
    if (warp == 0) {
      uint32_t c8[8], tot = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) { c8[q] = counts[lane * 8 + q]; tot += c8[q]; }
      uint32_t run = warp_incl_scan(tot, lane) - tot;
#pragma unroll
      for (int q = 0; q < 8; ++q) { s_base[lane * 8 + q] += run; run += c8[q]; }
    }
    __syncthreads();
    // the tile in digit order in shared memory, then written out in that
    // order: consecutive threads write consecutive slots of a digit's run
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      if (base + 32 * j + lane >= n) continue;
      const uint32_t lp = s_local[d[j]] + s_wcnt[warp][d[j]] + r[j];
      s_key[lp] = k[j];
      s_val[lp] = v[j];
    }
    __syncthreads();
    const uint32_t cnt = (uint32_t)min((uint64_t)kSortTile, n - (uint64_t)t * kSortTile);
    for (uint32_t i = threadIdx.x; i < cnt; i += kRadixThreads) {
      const uint32_t kk = s_key[i], vv = s_val[i];
      const uint32_t dd = dg(kk, vv, pass);
      const uint64_t pos = (uint64_t)s_base[dd] + (i - s_local[dd]);
      if (pos < n) {
        key_out[pos] = kk;
        val_out[pos] = vv;
      }
    }
    __syncthreads();  // shared arrays are reused by the next tile
  }
}

}  // namespace gsb
