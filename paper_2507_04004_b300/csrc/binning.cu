// Binning of the kept (Gaussian, tile) pairs into per-tile lists ordered by
// (depth key, Gaussian index) - the front-to-back order the compositing of
// Eq. rendered_rgb walks - without sorting any pair.
//
// The order of a tile's list is the order of its Gaussians' depth keys, and
// every Gaussian has one depth key per view.  So the visible (view, Gaussian)
// entries are sorted once, and everything after that is a stable scatter:
//   1. stable LSD radix sort of the visible entries by (view, depth key) -
//      four 8-bit passes on the key, one or two on the view, one kernel per
//      pass, the digit counts taken beside the scan of the (view, tile row)
//      buckets - then runs of equal keys put in index order
//      (k_counts_and_buckets, k_radix_pass, k_entry_order);
//   2. stable scatter of the sorted entries into (view, tile row) buckets,
//      one "row item" per tile row of an entry's box (k_entry_rows,
//      k_unit_scan, k_rows_scatter);
//   3. per row item the exact kept-tile span of Sec. "Fast Tile-based
//      Culling" (16 pixel-row chords) and per-tile counts (k_rows_count,
//      k_unit_scan), the tile ranges (k_scan_tiles);
//   4. stable scatter of the row items' kept tiles into the tile bins, which
//      writes each tile's Gaussian indices in order (k_rows_emit).
// Stable scatters: the input is cut into units (up to kEntryUnit sorted
// entries of one view, up to kRowUnit row items of one bucket), one warp per
// unit.  A unit's counts per output bin are scanned over the units of its
// segment in order, which gives each unit its first slot in every bin; inside
// a unit, a warp takes 32 inputs at a time and ranks each lane among the
// lower lanes that cover the same bin (per-warp lane masks in shared memory).
// Pairs and row items thus keep their input order, and no bin is sorted.
#include "gs_internal.h"
#include "radix.cuh"

namespace gsb {

constexpr int kScanThreads = 1024;
constexpr int kUnitWarps = 8;  // warps (units in flight) per CTA of the unit kernels


// Exclusive scan of count(i), i < n, by one CTA of NT threads: start[i] =
// sum of counts before i; returns the 64-bit total (to every thread).  Each
// warp owns a contiguous segment and walks it kScanLoads x 32 counts at a
// time (that many loads in flight per lane: one CTA's scan is bound by the
// round trips of its loads).
constexpr int kScanLoads = 8;
template <int NT, typename F>
__device__ unsigned long long block_scan(F count, uint32_t* start, int64_t n) {
  constexpr int NW = NT / 32;
  static_assert(NT % 32 == 0 && NW <= 32, "one warp scans the warps' sums");
  constexpr int L = kScanLoads;
  __shared__ unsigned long long wbase[NW + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = (n + NW - 1) / NW;
  const int64_t b = min(n, (int64_t)warp * seg), e = min(n, b + seg);
  unsigned long long s = 0;
  for (int64_t i0 = b; i0 < e; i0 += 32 * L) {
    unsigned long long c[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const int64_t i = i0 + 32 * j + lane;
      c[j] = i < e ? count(i) : 0u;
    }
#pragma unroll
    for (int j = 0; j < L; ++j) s += c[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if (lane == 0) wbase[warp] = s;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long v = lane < NW ? wbase[lane] : 0ull;
    unsigned long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane < NW) wbase[lane] = inc - v;
    if (lane == 31) wbase[NW] = inc;
  }
  __syncthreads();
  unsigned long long run = wbase[warp];
  for (int64_t i00 = b; i00 < e; i00 += 32 * L) {  // L loads in flight per lane, then L scans
    unsigned long long cc[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const int64_t i = i00 + 32 * j + lane;
      cc[j] = i < e ? count(i) : 0u;
    }
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const int64_t i = i00 + 32 * j + lane;
      const unsigned long long c = cc[j];
      unsigned long long inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
      }
      if (i < e) {
        const unsigned long long ex = run + inc - c;
        start[i] = ex > 0xffffffffull ? 0xffffffffu : (uint32_t)ex;
      }
      run += __shfl_sync(kFull, inc, 31);
    }
  }
  const unsigned long long total = wbase[NW];
  __syncthreads();
  return total;
}

// Units of n_seg segments of cnt(s) items (unit_count / unit_start): first[s]
// = first unit of segment s (first[n_seg] = total), seg[u] = segment of unit
// u, *total_out = total.  One CTA of NT threads; more than max_units units
// (not expected: the workspace is sized for the capacities checked before)
// flag an error.  Each warp writes the unit lists of 32 segments at a time,
// 32 consecutive units per store.
template <int NT, typename F>
__device__ void build_units(F cnt, int64_t n_seg, int unit_cap, int64_t max_units, uint32_t* first, uint32_t* seg,
                            uint32_t* total_out, uint32_t* status) {
  auto nu = [&](int64_t s) { return unit_count(cnt(s), unit_cap); };
  const unsigned long long total = block_scan<NT>(nu, first, n_seg);
  if (threadIdx.x == 0) {
    first[n_seg] = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    *total_out = total > (unsigned long long)max_units ? 0u : (uint32_t)total;
    if (total > (unsigned long long)max_units) atomicExch(status, (uint32_t)GS_ERR_CUDA);
  }
  __syncthreads();
  if (total > (unsigned long long)max_units) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t s0 = (int64_t)warp * 32; s0 < n_seg; s0 += NT) {
    uint32_t f = 0, k = 0;  // lane l: first unit and unit count of segment s0 + l
    if (s0 + lane < n_seg) {
      f = first[s0 + lane];
      k = nu(s0 + lane);
    }
    const int nq = (int)min((int64_t)32, n_seg - s0);
    for (int q = 0; q < nq; ++q) {
      const uint32_t fq = __shfl_sync(kFull, f, q), kq = __shfl_sync(kFull, k, q);
      for (uint32_t j = lane; j < kq; j += 32) seg[fq + j] = (uint32_t)(s0 + q);
    }
  }
}

// ---------------------------------------------------------------- buckets
// Bucket (view, tile row) ranges of the row items, capacity check, row units:
// one CTA of NT threads.
template <int NT>
__device__ void scan_buckets(const Ws& ws) {
  // The projection leaves each view's row-item counts as differences over the
  // tile rows (+1 at an entry's first row, -1 after its last, modulo 2^32):
  // a running sum per view, one warp per view, turns them into counts (up to
  // 8 x 32 rows loaded at once).
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ny = ws.tiles_y;
    for (int v = warp; v < ws.views; v += NT / 32) {
      uint32_t* c = ws.bucket_count + (int64_t)v * ny;
      uint32_t carry = 0;
      for (int t00 = 0; t00 < ny; t00 += 8 * 32) {
        uint32_t x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int ty = t00 + 32 * q + lane;
          x[q] = ty < ny ? c[ty] : 0u;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (t00 + 32 * q >= ny) break;
          const int ty = t00 + 32 * q + lane;
          const uint32_t inc = warp_incl_scan(x[q], lane) + carry;
          if (ty < ny) c[ty] = inc;
          carry = __shfl_sync(kFull, inc, 31);
        }
      }
    }
    __syncthreads();
  }
  const int64_t nb = (int64_t)ws.views * ws.tiles_y;
  const uint32_t* bc = ws.bucket_count;
  const unsigned long long total = block_scan<NT>([&](int64_t i) { return bc[i]; }, ws.bucket_start, nb);
  if (threadIdx.x == 0) {
    ws.counters[kRowCount] = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    if (total > (unsigned long long)ws.cap) {
      ws.counters[kPairsNeeded] = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
      ws.counters[kStatus] = (uint32_t)GS_ERR_CAPACITY;
    }
  }
  if (total > (unsigned long long)ws.cap) return;
  build_units<NT>([&](int64_t s) { return bc[s]; }, nb, kRowUnit, ws.units_r_max, ws.unit_first_r, ws.unit_seg_r,
                  ws.counters + kRowUnits, ws.counters + kStatus);
}

// ---------------------------------------------------------------- entry sort
// Digit of a visible entry (key = depth key bits, val = entry v*N + g) in
// pass p: bytes of the depth key for p < 4, then the bytes of the view.  LSD
// order makes the last pass the most significant: (view, depth key).
struct DepthDigit {
  uint32_t n_per_view;
  __device__ __forceinline__ uint32_t operator()(uint32_t key, uint32_t val, int pass) const {
    if (pass < 4) return (key >> (8 * pass)) & 255u;
    const uint32_t v = val / n_per_view;
    return (pass == 4 ? v : v >> 8) & 255u;
  }
};

// The depth sort's digit counts (all CTAs but the last) beside the bucket
// scan (the last CTA).  The two are independent, so the single-CTA scan runs
// next to the counting instead of as a launch of its own before it.  A
// capacity error the scan raises meanwhile leaves the counts harmless: the
// sort's passes and everything after them check the status word first.
__global__ void __launch_bounds__(kRadixThreads) k_counts_and_buckets(Ws ws, RadixScratch rs, DepthDigit dg,
                                                                      int passes) {
  if (blockIdx.x + 1 == gridDim.x) {
    scan_buckets<kRadixThreads>(ws);
    return;
  }
  radix_counts(rs, dg, passes, ws.vis_key, ws.visible, blockIdx.x, gridDim.x - 1);
}



// Runs of equal (view, depth key) put in Gaussian-index order, the sorted
// entries written to ws.sorted; first sorted entry of every view.  (The
// projection-order list in ws.visible is kept: the pose-only backward walks
// it.)
__global__ void __launch_bounds__(256) k_entry_order(Ws ws, const uint32_t* __restrict__ key,
                                                     const uint32_t* __restrict__ val) {
  if (ws.counters[kStatus] != 0) return;
  const uint64_t n = ws.counters[kVisibleCount];
  const uint32_t N = (uint32_t)ws.n;
  const int64_t V = ws.views;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  if (n == 0) {
    for (uint64_t u = tid; u <= (uint64_t)V; u += stride) ws.view_start[u] = 0;
    return;
  }
  for (uint64_t i = tid; i < n; i += stride) {
    const uint32_t k = key[i], e = val[i], v = e / N;
    auto same = [&](uint64_t j) { return key[j] == k && val[j] / N == v; };
    const bool prev = i > 0 && same(i - 1), next = i + 1 < n && same(i + 1);
    if (!prev && !next) {
      ws.sorted[i] = e;
    } else {
      uint64_t s = i, t = i + 1;
      while (s > 0 && same(s - 1)) --s;
      while (t < n && same(t)) ++t;
      uint32_t rank = 0;
      for (uint64_t j = s; j < t; ++j) rank += val[j] < e ? 1u : 0u;
      ws.sorted[s + rank] = e;
    }
    const int64_t vp = i > 0 ? (int64_t)(val[i - 1] / N) : -1;
    for (int64_t u = vp + 1; u <= (int64_t)v; ++u) ws.view_start[u] = (uint32_t)i;
    if (i + 1 == n)
      for (int64_t u = (int64_t)v + 1; u <= V; ++u) ws.view_start[u] = (uint32_t)n;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_entry_units(Ws ws) {
  if (ws.counters[kStatus] != 0) return;
  const uint32_t* vs = ws.view_start;
  build_units<kScanThreads>([&](int64_t s) { return vs[s + 1] - vs[s]; }, ws.views, kEntryUnit, ws.units_e_max,
                            ws.unit_first_e, ws.unit_seg_e, ws.counters + kEntryUnits, ws.counters + kStatus);
}

// ---------------------------------------------------------------- stable scatters
// Exclusive scan of unit counts over each segment's units, per bin, one warp
// per (segment, bin).  Tables are bin-major, table[x * stride + u], so a
// segment's units are contiguous in each bin's row: table[x][u] becomes the
// first slot of unit u in bin x relative to the bin's start.  totals (may be
// NULL) receives each (segment, bin) total; expect (may be NULL) holds totals
// to check against.
__global__ void __launch_bounds__(256) k_unit_scan(Ws ws, uint32_t* __restrict__ table, int64_t stride,
                                                   const uint32_t* __restrict__ first, int64_t n_seg, int bins,
                                                   uint32_t* __restrict__ totals, const uint32_t* __restrict__ expect) {
  if (ws.counters[kStatus] != 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (idx >= n_seg * bins) return;
  const int64_t s = idx / bins;
  const int x = (int)(idx - s * bins);
  const uint32_t u0 = first[s], u1 = first[s + 1];
  uint32_t* row = table + (int64_t)x * stride;
  uint32_t run = 0;
  for (uint32_t c0 = u0; c0 < u1; c0 += 128) {
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t u = c0 + 32 * j + lane;
      c[j] = u < u1 ? row[u] : 0u;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t u = c0 + 32 * j + lane;
      const uint32_t incl = warp_incl_scan(c[j], lane);
      if (u < u1) row[u] = run + incl - c[j];
      run += __shfl_sync(kFull, incl, 31);
    }
  }
  if (lane == 0) {
    if (totals) totals[s * bins + x] = run;
    if (expect && expect[s * bins + x] != run) atomicExch(ws.counters + kStatus, (uint32_t)GS_ERR_CUDA);
  }
}

// Row items per tile row of every entry unit (differences, then a prefix).
__global__ void __launch_bounds__(32 * kUnitWarps) k_entry_rows(Ws ws) {
  extern __shared__ uint32_t s_dyn[];
  if (ws.counters[kStatus] != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ny = ws.tiles_y;
  uint32_t* cnt = s_dyn + warp * (ny + 1);
  const uint32_t nu = ws.counters[kEntryUnits];
  for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < nu; u += gridDim.x * kUnitWarps) {
    const uint32_t v = ws.unit_seg_e[u];
    const uint32_t k = u - ws.unit_first_e[v];
    const uint32_t i0 = ws.view_start[v] + (uint32_t)unit_start(k, kEntryUnit);
    const uint32_t i1 = min(ws.view_start[v] + (uint32_t)unit_start(k + 1, kEntryUnit), ws.view_start[v + 1]);
    for (int t = lane; t <= ny; t += 32) cnt[t] = 0;
    __syncwarp();
    for (uint32_t i = i0 + lane; i < i1; i += 32) {
      const uint2 r = ws.rects[ws.sorted[i]];
      atomicAdd(cnt + (r.x >> 16), 1u);
      atomicSub(cnt + (r.y >> 16) + 1, 1u);
    }
    __syncwarp();
    uint32_t run = 0;
    for (int t0 = 0; t0 < ny; t0 += 32) {
      const int t = t0 + lane;
      const uint32_t x = warp_incl_scan(t < ny ? cnt[t] : 0u, lane) + run;
      if (t < ny) ws.unit_cnt_e[(int64_t)t * ws.units_e_max + u] = x;
      run = __shfl_sync(kFull, x, 31);
    }
    __syncwarp();
  }
}

// Stable scatter of one warp round: lane l's input (payload p_l, flag q_l)
// covers c_l consecutive bins from lo_l.  The round's (input, bin) pairs are
// enumerated in input order, 32 per sub-round, each lane finding its input by
// a binary search of the inputs' exclusive prefix counts (shuffles).  Inside
// a bin the pairs of one sub-round come from distinct inputs in lane order,
// and a later sub-round's from later inputs, so ranking the lanes of each bin
// within its sub-round (per-warp lane masks in shared memory) and advancing
// the bin's base after every sub-round keeps input order; all 32 lanes stay
// busy however unequal the inputs' bin counts are.
//   keep(p, q, bin): whether the pair takes a slot;
//   emit(p, bin, slot): writes it (slot = the bin's next free slot + rank).
template <class Keep, class Emit>
__device__ __forceinline__ void warp_stable_scatter(uint32_t lo, uint32_t c, uint32_t payload, uint32_t flag,
                                                    int lane, uint32_t* base, uint32_t* mask, Keep keep, Emit emit) {
  const unsigned lt = lanemask_lt(lane);
  const uint32_t incl = warp_incl_scan(c, lane);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  const uint32_t pre = incl - c;
  for (uint32_t f0 = 0; f0 < total; f0 += 32) {
    const uint32_t f = f0 + lane;
    int src = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint32_t p = __shfl_sync(kFull, pre, src + step);
      if (p <= f) src += step;
    }
    const uint32_t bin = __shfl_sync(kFull, lo, src) + (f - __shfl_sync(kFull, pre, src));
    const uint32_t ps = __shfl_sync(kFull, payload, src), qs = __shfl_sync(kFull, flag, src);
    const bool act = f < total && keep(ps, qs, bin);
    if (act) atomicOr(mask + bin, 1u << lane);
    __syncwarp();
    uint32_t m = 0, rank = 0;
    if (act) {
      m = mask[bin];
      rank = __popc(m & lt);
      emit(ps, bin, base[bin] + rank);
    }
    __syncwarp();
    if (act && rank == 0) {  // lowest lane of this bin in the sub-round
      base[bin] += __popc(m);
      mask[bin] = 0;
    }
    __syncwarp();
  }
}

// Sorted entries -> row items, grouped by (view, tile row), in entry order.
__global__ void __launch_bounds__(32 * kUnitWarps) k_rows_scatter(Ws ws) {
  extern __shared__ uint32_t s_dyn[];
  if (ws.counters[kStatus] != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ny = ws.tiles_y;
  uint32_t* base = s_dyn + warp * 3 * ny;
  uint32_t* end = base + ny;
  uint32_t* mask = end + ny;
  const uint32_t nu = ws.counters[kEntryUnits];
  for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < nu; u += gridDim.x * kUnitWarps) {
    const uint32_t v = ws.unit_seg_e[u];
    const uint32_t k = u - ws.unit_first_e[v];
    const uint32_t i0 = ws.view_start[v] + (uint32_t)unit_start(k, kEntryUnit);
    const uint32_t i1 = min(ws.view_start[v] + (uint32_t)unit_start(k + 1, kEntryUnit), ws.view_start[v + 1]);
    for (int t = lane; t < ny; t += 32) {
      const int64_t b = (int64_t)v * ny + t;
      const uint32_t bs = ws.bucket_start[b];
      base[t] = bs + ws.unit_cnt_e[(int64_t)t * ws.units_e_max + u];
      end[t] = bs + ws.bucket_count[b];
      mask[t] = 0;
    }
    __syncwarp();
    uint32_t ne = 0;  // next round's entry and box, loaded ahead
    uint2 nr = make_uint2(1u, 0u);
    if (i0 + lane < i1) {
      ne = ws.sorted[i0 + lane];
      nr = ws.rects[ne];
    }
    for (uint32_t r0 = i0; r0 < i1; r0 += 32) {
      const uint32_t e = ne;
      const uint32_t y0 = nr.x >> 16;
      const uint32_t c = r0 + lane < i1 ? (nr.y >> 16) - y0 + 1 : 0u;
      if (r0 + 32 + lane < i1) {
        ne = ws.sorted[r0 + 32 + lane];
        nr = ws.rects[ne];
      }
      warp_stable_scatter(
          y0, c, e, 0u, lane, base, mask, [](uint32_t, uint32_t, uint32_t) { return true; },
          [&](uint32_t es, uint32_t row, uint32_t pos) {
            if (pos < end[row]) ws.row_items[pos] = es;
            else atomicExch(ws.counters + kStatus, (uint32_t)GS_ERR_CUDA);
          });
    }
  }
}

// Kept-tile span of every row item (Sec. "Fast Tile-based Culling": the
// exact chords of the 16 pixel rows) and pairs per tile of every row unit.
__global__ void __launch_bounds__(32 * kUnitWarps) k_rows_count(Ws ws) {
  extern __shared__ uint32_t s_dyn[];
  if (ws.counters[kStatus] != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nx = ws.tiles_x;
  uint32_t* cnt = s_dyn + warp * (nx + 1);
  const uint32_t nu = ws.counters[kRowUnits];
  for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < nu; u += gridDim.x * kUnitWarps) {
    const uint32_t b = ws.unit_seg_r[u];
    const int ty = (int)(b % (uint32_t)ws.tiles_y);
    const uint32_t bs = ws.bucket_start[b];
    const uint32_t k = u - ws.unit_first_r[b];
    const uint32_t i0 = bs + (uint32_t)unit_start(k, kRowUnit);
    const uint32_t i1 = min(bs + (uint32_t)unit_start(k + 1, kRowUnit), bs + ws.bucket_count[b]);
    for (int t = lane; t <= nx; t += 32) cnt[t] = 0;
    __syncwarp();
    // the next item's record is loaded while this one's chords are evaluated
    uint32_t i = i0 + lane;
    float4 n0 = make_float4(0.f, 0.f, 1.f, 0.f), n1 = make_float4(1.f, 0.f, 0.f, 0.f);
    if (i < i1) {
      const int64_t e = ws.row_items[i];
      n0 = ws.records[3 * e];
      n1 = ws.records[3 * e + 1];
    }
    for (; i < i1; i += 32) {
      const Ellipse el = make_ellipse(n0, n1);
      if (i + 32 < i1) {
        const int64_t e = ws.row_items[i + 32];
        n0 = ws.records[3 * e];
        n1 = ws.records[3 * e + 1];
      }
      const RowSpan sp = row_span(el, ty, ws.width, ws.height);
      ws.row_span[i] = pack_span(sp);
      if (sp.lo > sp.hi) continue;
      if (!sp.gap) {
        atomicAdd(cnt + sp.lo, 1u);
        atomicSub(cnt + sp.hi + 1, 1u);
      } else {
        for (int tx = sp.lo; tx <= sp.hi; ++tx)
          if (tile_kept(el, tx, ty, ws.width, ws.height)) {
            atomicAdd(cnt + tx, 1u);
            atomicSub(cnt + tx + 1, 1u);
          }
      }
    }
    __syncwarp();
    uint32_t run = 0;
    for (int t0 = 0; t0 < nx; t0 += 32) {
      const int t = t0 + lane;
      const uint32_t x = warp_incl_scan(t < nx ? cnt[t] : 0u, lane) + run;
      if (t < nx) ws.unit_cnt_r[(int64_t)t * ws.units_r_max + u] = x;
      run = __shfl_sync(kFull, x, 31);
    }
    __syncwarp();
  }
}

// Tile ranges of the pairs (exclusive scan of the per-tile counts) and the
// capacity check.  Counts fit in 32 bits; the total is checked in 64 bits.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(Ws ws) {
  if (ws.counters[kStatus] != 0) return;
  const uint32_t* tc = ws.tile_count;
  const unsigned long long total =
      block_scan<kScanThreads>([&](int64_t i) { return tc[i]; }, ws.tile_start, (int64_t)ws.views * ws.tiles_per_view);
  if (threadIdx.x == 0) {
    ws.counters[kPairsNeeded] = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    if (total > (unsigned long long)ws.cap) ws.counters[kStatus] = (uint32_t)GS_ERR_CAPACITY;
  }
}

// Row items -> the Gaussian index of every kept (Gaussian, tile) pair in its
// tile's bin, in row-item order, i.e. (depth key, index) order.
__global__ void __launch_bounds__(32 * kUnitWarps) k_rows_emit(Ws ws) {
  extern __shared__ uint32_t s_dyn[];
  if (ws.counters[kStatus] != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nx = ws.tiles_x;
  uint32_t* base = s_dyn + warp * 3 * nx;
  uint32_t* end = base + nx;
  uint32_t* mask = end + nx;
  const int64_t N = ws.n;
  const uint32_t nu = ws.counters[kRowUnits];
  for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < nu; u += gridDim.x * kUnitWarps) {
    const uint32_t b = ws.unit_seg_r[u];
    const int ty = (int)(b % (uint32_t)ws.tiles_y);
    const int64_t vN = (int64_t)(b / (uint32_t)ws.tiles_y) * N;
    const uint32_t bs = ws.bucket_start[b];
    const uint32_t k = u - ws.unit_first_r[b];
    const uint32_t i0 = bs + (uint32_t)unit_start(k, kRowUnit);
    const uint32_t i1 = min(bs + (uint32_t)unit_start(k + 1, kRowUnit), bs + ws.bucket_count[b]);
    for (int x = lane; x < nx; x += 32) {
      const int64_t t = (int64_t)b * nx + x;
      const uint32_t ts = ws.tile_start[t];
      base[x] = ts + ws.unit_cnt_r[(int64_t)x * ws.units_r_max + u];
      end[x] = ts + ws.tile_count[t];
      mask[x] = 0;
    }
    __syncwarp();
    uint32_t nspan = 0xfffu, nitem = 0;  // next round's span and item, loaded ahead
    if (i0 + lane < i1) {
      nspan = ws.row_span[i0 + lane];
      nitem = ws.row_items[i0 + lane];
    }
    for (uint32_t r0 = i0; r0 < i1; r0 += 32) {
      const RowSpan sp = unpack_span(nspan);
      const uint32_t e = nitem;
      const uint32_t c = sp.lo <= sp.hi ? (uint32_t)(sp.hi - sp.lo + 1) : 0u;
      const uint32_t lo = sp.lo <= sp.hi ? (uint32_t)sp.lo : 0u;
      if (r0 + 32 + lane < i1) {
        nspan = ws.row_span[r0 + 32 + lane];
        nitem = ws.row_items[r0 + 32 + lane];
      } else {
        nspan = 0xfffu;
      }
      warp_stable_scatter(
          lo, c, e, sp.gap ? 1u : 0u, lane, base, mask,
          [&](uint32_t es, uint32_t gap, uint32_t x) {
            // a span with a gap (very thin tilted ellipses): its tiles are tested exactly
            if (!gap) return true;
            const Ellipse el = make_ellipse(ws.records[3 * (int64_t)es], ws.records[3 * (int64_t)es + 1]);
            return tile_kept(el, (int)x, ty, ws.width, ws.height);
          },
          [&](uint32_t es, uint32_t x, uint32_t pos) {
            if (pos < end[x]) ws.sorted_ids[pos] = (uint32_t)((int64_t)es - vN);
            else atomicExch(ws.counters + kStatus, (uint32_t)GS_ERR_CUDA);
          });
    }
  }
}

cudaError_t launch_bin_sort(const Ws& ws, cudaStream_t st) {
  cudaError_t err;
  auto done = [&](void) { trace_end(st); return cudaGetLastError(); };

  // 1. entries sorted by (view, depth key), then index inside equal keys
  const int64_t E = (int64_t)ws.views * ws.n;
  const int passes = depth_sort_passes(ws.views);
  // the sort's host view of its scratch (device pointers and the entry count's slot)
  RadixScratch rs;
  rs.n = ws.counters + kVisibleCount;
  rs.status = ws.counters + kStatus;
  rs.counts = ws.radix_status;
  rs.tiles = ws.radix_status + 6 * 256;
  rs.tickets = ws.counters + kRadixTicket;
  rs.tiles_max = ws.radix_tiles_max;
  const DepthDigit dg{(uint32_t)ws.n};
  // digit counts from zero; with them the bucket ranges and row units
  if ((err = cudaMemsetAsync(ws.radix_status, 0, 6 * 256 * sizeof(uint32_t), st)) != cudaSuccess) return err;
  trace_begin(kKDepthHist, st);
  k_counts_and_buckets<<<sm_count() * 4 + 1, kRadixThreads, 0, st>>>(ws, rs, dg, passes);
  if ((err = done()) != cudaSuccess) return err;
  const uint32_t* key = ws.vis_key;
  const uint32_t* val = ws.visible;
  for (int p = 0; p < passes; ++p) {
    uint32_t* ko = ws.sort_key + (p & 1) * E;
    uint32_t* vo = ws.sort_val + (p & 1) * E;
    trace_begin(kKDepthScatter, st);
    k_radix_pass<<<sm_count() * 4, kRadixThreads, 0, st>>>(rs, dg, p, key, val, ko, vo);
    if ((err = done()) != cudaSuccess) return err;
    key = ko;
    val = vo;
  }
  trace_begin(kKEntryOrder, st);
  k_entry_order<<<sm_count() * 4, 256, 0, st>>>(ws, key, val);
  if ((err = done()) != cudaSuccess) return err;
  trace_begin(kKEntryUnits, st);
  k_entry_units<<<1, kScanThreads, 0, st>>>(ws);
  if ((err = done()) != cudaSuccess) return err;

  // 2. row items by (view, tile row), entry order inside
  const unsigned ugrid = (unsigned)sm_count() * 8;
  const size_t smem_er = (size_t)kUnitWarps * (ws.tiles_y + 1) * sizeof(uint32_t);
  trace_begin(kKEntryRows, st);
  k_entry_rows<<<ugrid, 32 * kUnitWarps, smem_er, st>>>(ws);
  if ((err = done()) != cudaSuccess) return err;
  const int64_t ne = (int64_t)ws.views * ws.tiles_y;
  trace_begin(kKUnitScan, st);
  k_unit_scan<<<(unsigned)((ne + 7) / 8), 256, 0, st>>>(ws, ws.unit_cnt_e, ws.units_e_max, ws.unit_first_e, ws.views,
                                                        ws.tiles_y, nullptr, ws.bucket_count);
  if ((err = done()) != cudaSuccess) return err;
  const size_t smem_rs = (size_t)kUnitWarps * 3 * ws.tiles_y * sizeof(uint32_t);
  trace_begin(kKScatterRows, st);
  k_rows_scatter<<<ugrid, 32 * kUnitWarps, smem_rs, st>>>(ws);
  if ((err = done()) != cudaSuccess) return err;

  // 3. kept-tile spans, tile counts and ranges
  const size_t smem_rc = (size_t)kUnitWarps * (ws.tiles_x + 1) * sizeof(uint32_t);
  trace_begin(kKRowsCount, st);
  k_rows_count<<<ugrid, 32 * kUnitWarps, smem_rc, st>>>(ws);
  if ((err = done()) != cudaSuccess) return err;
  const int64_t nt = (int64_t)ws.views * ws.tiles_per_view;
  trace_begin(kKUnitScan, st);
  k_unit_scan<<<(unsigned)((nt + 7) / 8), 256, 0, st>>>(ws, ws.unit_cnt_r, ws.units_r_max, ws.unit_first_r,
                                                        (int64_t)ws.views * ws.tiles_y, ws.tiles_x, ws.tile_count,
                                                        nullptr);
  if ((err = done()) != cudaSuccess) return err;
  trace_begin(kKScan, st);
  k_scan_tiles<<<1, kScanThreads, 0, st>>>(ws);
  if ((err = done()) != cudaSuccess) return err;

  // 4. the tile bins, filled in order
  const size_t smem_em = (size_t)kUnitWarps * 3 * ws.tiles_x * sizeof(uint32_t);
  trace_begin(kKRowsEmit, st);
  k_rows_emit<<<ugrid, 32 * kUnitWarps, smem_em, st>>>(ws);
  return done();
}

}  // namespace gsb
