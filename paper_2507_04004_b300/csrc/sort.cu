// Tile binning and sorting of (Gaussian, tile) pairs by the 64-bit key
// (tile id << 32 | depth key bits), ties by Gaussian index.
//
// The sort is a two-level most-significant-digit radix sort: the first digit
// is the whole (view, tile) id, done as a counting sort (per-tile counts from
// the projection, an exclusive scan here, and binning by per-tile cursors in
// the emit kernel); the remaining 64 bits (depth key bits << 32 | Gaussian
// index) are unique inside a bin and are sorted per tile in shared memory
// (by size class: warp bitonic, CTA radix in a small or a medium CTA, bitonic
// network with a merge of sorted runs for the rare bins longer than that).  The result for each tile is its Gaussians in
// front-to-back order, as the compositing of Eq. rendered_rgb needs.
#include "gs_internal.h"

namespace gsb {

constexpr int kScanThreads = 1024;
constexpr int kLongCap = 16384;      // keys sorted by a 1024-thread CTA (128 KB)

// Exclusive scan of n counts by one CTA: start[i] = sum of counts before i,
// cursor[i] = start[i]; returns the 64-bit total (to every thread).  Each
// warp owns a contiguous segment and walks it 32 consecutive counts at a
// time (coalesced), with shuffle scans; a scan over the warp totals links
// the segments.
__device__ unsigned long long block_scan(const uint32_t* count, uint32_t* start, uint32_t* cursor, int64_t n) {
  constexpr int NW = kScanThreads / 32;
  __shared__ unsigned long long wbase[NW + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = (n + NW - 1) / NW;
  const int64_t b = min(n, (int64_t)warp * seg), e = min(n, b + seg);
  unsigned long long s = 0;
#pragma unroll 4
  for (int64_t i = b + lane; i < e; i += 32) s += count[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if (lane == 0) wbase[warp] = s;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long v = wbase[lane];  // NW == 32
    unsigned long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    wbase[lane] = inc - v;
    if (lane == 31) wbase[NW] = inc;
  }
  __syncthreads();
  unsigned long long run = wbase[warp];
#pragma unroll 2
  for (int64_t i0 = b; i0 < e; i0 += 32) {
    const int64_t i = i0 + lane;
    const unsigned long long c = i < e ? count[i] : 0u;
    unsigned long long inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    if (i < e) {
      const unsigned long long ex = run + inc - c;
      const uint32_t st = ex > 0xffffffffull ? 0xffffffffu : (uint32_t)ex;
      start[i] = st;
      cursor[i] = st;
    }
    run += __shfl_sync(kFull, inc, 31);
  }
  const unsigned long long total = wbase[NW];
  __syncthreads();
  return total;
}

// Bucket (view, tile row) ranges of the row items; capacity check.
__global__ void __launch_bounds__(kScanThreads) k_scan_buckets(Ws ws) {
  // The projection leaves each view's row-item counts as differences over the
  // tile rows (+1 at an entry's first row, -1 after its last, modulo 2^32):
  // a running sum per view, one warp per view, turns them into counts.
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int v = warp; v < ws.views; v += kScanThreads / 32) {
      uint32_t* c = ws.bucket_count + (int64_t)v * ws.tiles_y;
      uint32_t carry = 0;
      for (int t0 = 0; t0 < ws.tiles_y; t0 += 32) {
        const int ty = t0 + lane;
        uint32_t x = ty < ws.tiles_y ? c[ty] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, x, o);
          if (lane >= o) x += y;
        }
        x += carry;
        if (ty < ws.tiles_y) c[ty] = x;
        carry = __shfl_sync(kFull, x, 31);
      }
    }
    __syncthreads();
  }
  const unsigned long long total =
      block_scan(ws.bucket_count, ws.bucket_start, ws.bucket_cursor, (int64_t)ws.views * ws.tiles_y);
  if (threadIdx.x == 0) {
    ws.counters[kRowCount] = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    if (total > (unsigned long long)ws.cap) {
      ws.counters[kPairsNeeded] = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
      ws.counters[kStatus] = (uint32_t)GS_ERR_CAPACITY;
    }
  }
}

// Tile ranges of the pairs (exclusive scan of the per-tile counts), capacity
// check, cursor initialisation.  Counts fit in 32 bits; the total is checked
// in 64 bits.
__global__ void __launch_bounds__(kScanThreads) k_scan(Ws ws) {
  if (ws.counters[kStatus] != 0) return;
  const unsigned long long total =
      block_scan(ws.tile_count, ws.tile_start, ws.tile_cursor, (int64_t)ws.views * ws.tiles_per_view);
  if (threadIdx.x == 0) {
    ws.counters[kPairsNeeded] = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    ws.counters[kLongCount] = 0;
    ws.counters[kMediumCount] = 0;
    if (total > (unsigned long long)ws.cap) ws.counters[kStatus] = (uint32_t)GS_ERR_CAPACITY;
  }
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// In-place ascending bitonic sort of s[0, np2) by the whole CTA.
__device__ __forceinline__ void bitonic_smem(unsigned long long* s, int np2) {
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < (np2 >> 1); i += blockDim.x) {
        const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));  // j is a power of two
        const int hi = lo + j;
        const bool up = (lo & k) == 0;
        const unsigned long long a = s[lo], c = s[hi];
        if ((a > c) == up) { s[lo] = c; s[hi] = a; }
      }
      __syncthreads();
    }
  }
}

// Sort one tile's keys held in shared memory and write the Gaussian indices.
__device__ __forceinline__ void sort_tile_smem(const Ws& ws, unsigned long long* s, uint32_t start, int cnt) {
  const int np2 = next_pow2(cnt);
  for (int i = threadIdx.x; i < np2; i += blockDim.x) s[i] = i < cnt ? ws.keys[start + i] : ~0ull;
  __syncthreads();
  bitonic_smem(s, np2);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) ws.sorted_ids[start + i] = (uint32_t)(s[i] & 0xffffffffull);
  __syncthreads();
}

// Register bitonic sort of one bin of n <= 32 E keys by one warp.  Element
// i = e * 32 + lane lives in register v[e] of that lane: compare distances
// j < 32 exchange across lanes with shuffles, larger ones stay in-thread.
// Stage loops run at run time (small code); only the loops over a thread's E
// elements are unrolled.
template <int E, int JE>
__device__ __forceinline__ void warp_sort_intra(unsigned long long* v, int k, int lane) {
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (e & JE) continue;
    const int f = e | JE;
    const bool asc = ((e * 32 + lane) & k) == 0;
    const unsigned long long a = v[e], b = v[f];
    const bool swap = (a > b) == asc;
    v[e] = swap ? b : a;
    v[f] = swap ? a : b;
  }
}

template <int E>
__device__ __forceinline__ void warp_sort_bin(const Ws& ws, uint32_t start, int n, int lane) {
  constexpr int N = 32 * E;
  unsigned long long v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    v[e] = i < n ? ws.keys[start + i] : ~0ull;
  }
#pragma unroll 1
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll 1
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        switch (j >> 5) {
          case 1: warp_sort_intra<E, 1>(v, k, lane); break;
          case 2: warp_sort_intra<E, (E > 2 ? 2 : 1)>(v, k, lane); break;
          case 4: warp_sort_intra<E, (E > 4 ? 4 : 1)>(v, k, lane); break;
          case 8: warp_sort_intra<E, (E > 8 ? 8 : 1)>(v, k, lane); break;
          default: warp_sort_intra<E, (E > 16 ? 16 : 1)>(v, k, lane); break;
        }
      } else {
        const bool lower = (lane & j) == 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const bool asc = ((e * 32 + lane) & k) == 0;
          const unsigned long long b = __shfl_xor_sync(kFull, v[e], j);
          const bool keep_min = lower == asc;
          v[e] = keep_min ? (v[e] < b ? v[e] : b) : (v[e] < b ? b : v[e]);
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    if (i < n) ws.sorted_ids[start + i] = (uint32_t)(v[e] & 0xffffffffull);
  }
}

// CTA radix sort of one bin held in shared memory: stable LSD radix sort on
// the 32-bit depth key (8-bit digits; a pass whose digit is the same for
// every key is skipped), each warp ranking its contiguous share with
// __match_any_sync, then short runs of equal keys ordered by (key, Gaussian
// index).  NT threads, bins of up to CAP keys.
template <int NT, int CAP>
struct RadixSmem {
  uint32_t key[2][CAP];
  uint32_t val[2][CAP];
  uint32_t hist[NT / 32][256];
  uint32_t tot[256];
  int skip[8];  // one flag per pass: no thread can still be reading a reset flag
};

template <int NT, int CAP>
__device__ void cta_radix_bin(const Ws& ws, uint32_t start, int n, RadixSmem<NT, CAP>& sm) {
  constexpr int NW = NT / 32;
  auto& s_key = sm.key;
  auto& s_val = sm.val;
  auto& s_hist = sm.hist;
  auto& s_tot = sm.tot;
  auto& s_skip = sm.skip;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < n; i += NT) {
    const unsigned long long k = ws.keys[start + i];
    s_key[0][i] = (uint32_t)(k >> 32);
    s_val[0][i] = (uint32_t)(k & 0xffffffffull);
  }
  if (threadIdx.x < 8) s_skip[threadIdx.x] = 0;
  const int chunk = ((n + NW - 1) / NW + 31) & ~31;  // each warp's contiguous share, whole rounds
  const int w0 = min(n, warp * chunk), w1 = min(n, w0 + chunk);
  int src = 0, pass = 0;
  // one stable LSD pass on the 8-bit digit at `shift`
  auto radix_pass = [&](int shift) {
    for (int i = threadIdx.x; i < NW * 256; i += NT) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    for (int i = w0 + lane; i < w1; i += 32) atomicAdd(&s_hist[warp][(s_key[src][i] >> shift) & 255u], 1u);
    __syncthreads();
    {
      // digit-major exclusive scan: offsets[w][d] = sum_{d' < d} tot[d'] + sum_{w' < w} hist[w'][d]
      for (int d = threadIdx.x; d < 256; d += NT) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint32_t h = s_hist[w][d];
          s_hist[w][d] = run;
          run += h;
        }
        s_tot[d] = run;
        if (run == (uint32_t)n) s_skip[pass] = 1;
      }
    }
    __syncthreads();
    if (s_skip[pass]) {  // every key has this digit: the pass keeps the order
      ++pass;
      return;
    }
    {
      // exclusive scan of s_tot over the 256 digits (one warp)
      if (warp == 0) {
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { v[q] = s_tot[lane * 8 + q]; sum += v[q]; }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, inc, o);
          if (lane >= o) inc += y;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int q = 0; q < 8; ++q) { const uint32_t c = v[q]; s_tot[lane * 8 + q] = run; run += c; }
      }
      __syncthreads();
      for (int d = threadIdx.x; d < 256; d += NT)
#pragma unroll
        for (int w = 0; w < NW; ++w) s_hist[w][d] += s_tot[d];
    }
    __syncthreads();
    const int dst = src ^ 1;
    for (int base = w0; base < w1; base += 32) {
      const int i = base + lane;
      const unsigned active = __ballot_sync(kFull, i < w1);
      if (i < w1) {
        const uint32_t key = s_key[src][i];
        const uint32_t dg = (key >> shift) & 255u;
        const unsigned peers = __match_any_sync(active, dg);
        const uint32_t pos = s_hist[warp][dg] + __popc(peers & ((1u << lane) - 1u));
        s_key[dst][pos] = key;
        s_val[dst][pos] = s_val[src][i];
        __syncwarp(active);
        if (lane == __ffs(peers) - 1) s_hist[warp][dg] += __popc(peers);
      }
      __syncwarp();
    }
    src = dst;
    __syncthreads();
    ++pass;
  };
  // Two passes order the bin by the top 16 bits of the depth key; runs that
  // share those bits are then finished by ranking on (key, index).  A run
  // longer than 32 keys (near-constant depth) sends the bin through all four
  // passes instead, so the fix-up stays short.
  radix_pass(16);
  radix_pass(24);
  if (threadIdx.x == 0) s_tot[0] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += NT) {
    const uint32_t hi = s_key[src][i] >> 16;
    if (i == 0 || (s_key[src][i - 1] >> 16) != hi) {
      int e = i + 1;
      while (e < n && (s_key[src][e] >> 16) == hi && e - i <= 32) ++e;
      if (e - i > 32) atomicMax(&s_tot[0], (uint32_t)(e - i));
    }
  }
  __syncthreads();
  const bool full = s_tot[0] > 32;
  __syncthreads();
  if (full) {
    radix_pass(0);
    radix_pass(8);
    radix_pass(16);
    radix_pass(24);
  }
  const uint32_t mask = full ? 0xffffffffu : 0xffff0000u;
  // Runs of equal (masked) keys are finished in parallel: each key's place in
  // its run is the number of the run's keys below it in (key, Gaussian
  // index) order (all distinct), so it is written straight to its sorted slot.
  for (int i = threadIdx.x; i < n; i += NT) {
    const uint32_t ka = s_key[src][i], va = s_val[src][i];
    const uint32_t k = ka & mask;
    int s0 = i, e = i + 1;
    while (s0 > 0 && (s_key[src][s0 - 1] & mask) == k) --s0;
    while (e < n && (s_key[src][e] & mask) == k) ++e;
    int rank = 0;
    if (e - s0 > 1)
      for (int b = s0; b < e; ++b) {
        const uint32_t kb = s_key[src][b];
        rank += (kb < ka || (kb == ka && s_val[src][b] < va)) ? 1 : 0;
      }
    ws.sorted_ids[start + s0 + rank] = va;
  }
}

// Bins are sorted by size class: up to 64 keys by one warp (register bitonic
// on the full 64-bit key), up to kSmallCap by a kSmallThreads-thread CTA per
// bin (small shared memory, so many bins share an SM), up to kMediumCap by a
// persistent kMediumThreads-thread CTA over the medium list (filled from the
// end of long_tiles), longer ones by k_sort_long.
constexpr int kSmallThreads = 128, kSmallCap = 768;
constexpr int kMediumThreads = 256, kMediumCap = 2048;
constexpr int kMediumPerSm = 5;  // resident CTAs per SM (shared memory: 41 KB each)

__global__ void __launch_bounds__(kSmallThreads) k_sort_small(Ws ws) {
  __shared__ RadixSmem<kSmallThreads, kSmallCap> sm;
  if (ws.counters[kStatus] != 0) return;
  const int64_t t = blockIdx.x;
  const int n = (int)ws.tile_count[t];
  if (n == 0) return;
  const uint32_t start = ws.tile_start[t];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (n > kMediumCap) {
    if (threadIdx.x == 0) ws.long_tiles[atomicAdd(ws.counters + kLongCount, 1u)] = (uint32_t)t;
    return;
  }
  if (n > kSmallCap) {
    const int64_t ntiles = (int64_t)ws.views * ws.tiles_per_view;
    if (threadIdx.x == 0) ws.long_tiles[ntiles - 1 - atomicAdd(ws.counters + kMediumCount, 1u)] = (uint32_t)t;
    return;
  }
  if (n <= 64) {
    if (warp == 0) {
      if (n <= 32) warp_sort_bin<1>(ws, start, n, lane);
      else warp_sort_bin<2>(ws, start, n, lane);
    }
    return;
  }
  cta_radix_bin<kSmallThreads, kSmallCap>(ws, start, n, sm);
}

__global__ void __launch_bounds__(kMediumThreads) k_sort_medium(Ws ws) {
  // over 48 KB: dynamic shared memory (the launch raises the limit)
  extern __shared__ __align__(16) unsigned char s_medium[];
  auto& sm = *reinterpret_cast<RadixSmem<kMediumThreads, kMediumCap>*>(s_medium);
  if (ws.counters[kStatus] != 0) return;
  const int64_t ntiles = (int64_t)ws.views * ws.tiles_per_view;
  const uint32_t nm = ws.counters[kMediumCount];
  for (uint32_t li = blockIdx.x; li < nm; li += gridDim.x) {
    const int64_t t = ws.long_tiles[ntiles - 1 - li];
    cta_radix_bin<kMediumThreads, kMediumCap>(ws, ws.tile_start[t], (int)ws.tile_count[t], sm);
    __syncthreads();  // the next bin reuses the buffers and flags
  }
}

// Merge-path split: number of elements of A among the first d outputs of
// merge(A, B) (keys are unique).
__device__ __forceinline__ int merge_split(const unsigned long long* A, int la, const unsigned long long* B, int lb,
                                           int d) {
  int lo = max(0, d - lb), hi = min(d, la);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (A[mid] < B[d - mid - 1]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Long tiles: one 1024-thread CTA per tile.  Up to kLongCap keys are sorted
// in shared memory; longer bins are sorted in kLongCap chunks and the sorted
// runs merged pairwise (merge path) between keys and keys_alt.
__global__ void __launch_bounds__(1024) k_sort_long(Ws ws) {
  extern __shared__ unsigned long long sl[];
  if (ws.counters[kStatus] != 0) return;
  const uint32_t nl = ws.counters[kLongCount];
  for (uint32_t li = blockIdx.x; li < nl; li += gridDim.x) {
    const uint32_t t = ws.long_tiles[li];
    const int cnt = (int)ws.tile_count[t];
    const uint32_t start = ws.tile_start[t];
    if (cnt <= kLongCap) {
      sort_tile_smem(ws, sl, start, cnt);
      continue;
    }
    // sort chunks in place
    for (int c0 = 0; c0 < cnt; c0 += kLongCap) {
      const int m = min(kLongCap, cnt - c0);
      const int np2 = next_pow2(m);
      for (int i = threadIdx.x; i < np2; i += blockDim.x) sl[i] = i < m ? ws.keys[start + c0 + i] : ~0ull;
      __syncthreads();
      bitonic_smem(sl, np2);
      for (int i = threadIdx.x; i < m; i += blockDim.x) ws.keys[start + c0 + i] = sl[i];
      __syncthreads();
    }
    unsigned long long* src = ws.keys + start;
    unsigned long long* dst = ws.keys_alt + start;
    for (int run = kLongCap; run < cnt; run <<= 1) {
      for (int lo = 0; lo < cnt; lo += 2 * run) {
        const int mid = min(cnt, lo + run), hi = min(cnt, lo + 2 * run);
        const unsigned long long* A = src + lo;
        const unsigned long long* B = src + mid;
        const int la = mid - lo, lb = hi - mid, m = hi - lo;
        const int per = (m + blockDim.x - 1) / blockDim.x;
        const int d0 = min(m, (int)threadIdx.x * per), d1 = min(m, d0 + per);
        int ia = merge_split(A, la, B, lb, d0);
        int ib = d0 - ia;
        for (int d = d0; d < d1; ++d) {
          const bool takeA = ia < la && (ib >= lb || A[ia] < B[ib]);
          dst[lo + d] = takeA ? A[ia++] : B[ib++];
        }
      }
      __syncthreads();
      unsigned long long* tmp = src; src = dst; dst = tmp;
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) ws.sorted_ids[start + i] = (uint32_t)(src[i] & 0xffffffffull);
    __syncthreads();
  }
}

cudaError_t launch_rows(const Ws& ws, int phase, cudaStream_t st);

cudaError_t launch_bin_sort(const Ws& ws, cudaStream_t st) {
  trace_begin(kKScanBuckets, st);
  k_scan_buckets<<<1, kScanThreads, 0, st>>>(ws);
  trace_end(st);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if ((err = launch_rows(ws, 0, st)) != cudaSuccess) return err;
  if ((err = launch_rows(ws, 1, st)) != cudaSuccess) return err;
  trace_begin(kKScan, st);
  k_scan<<<1, kScanThreads, 0, st>>>(ws);
  trace_end(st);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if ((err = launch_rows(ws, 2, st)) != cudaSuccess) return err;
  const unsigned ntiles = (unsigned)((int64_t)ws.views * ws.tiles_per_view);
  trace_begin(kKSortSmall, st);
  k_sort_small<<<ntiles, kSmallThreads, 0, st>>>(ws);
  trace_end(st);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const int medium_smem = (int)sizeof(RadixSmem<kMediumThreads, kMediumCap>);
  err = cudaFuncSetAttribute(k_sort_medium, cudaFuncAttributeMaxDynamicSharedMemorySize, medium_smem);
  if (err != cudaSuccess) return err;
  trace_begin(kKSortMedium, st);
  k_sort_medium<<<sm_count() * kMediumPerSm, kMediumThreads, medium_smem, st>>>(ws);
  trace_end(st);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const size_t smem = (size_t)kLongCap * sizeof(unsigned long long);
  err = cudaFuncSetAttribute(k_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  trace_begin(kKSortLong, st);
  k_sort_long<<<sm_count(), 1024, smem, st>>>(ws);
  trace_end(st);
  return cudaGetLastError();
}

}  // namespace gsb
