// scan.cuh - the record scan shared by the two bin/sort paths (binsort.cu, onesweep.cu): a
// single-pass scan of tiles_touched with decoupled look-back, and the helpers it and the
// tile scan use. Included inside each file's anonymous namespace.
#pragma once

#include "fgs_internal.cuh"

namespace fgs {
namespace {

constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 2ull << 62;
constexpr uint64_t LB_VAL = (1ull << 62) - 1;

// exclusive scan over a block of 256 threads; returns the block total in *total
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t *s_warp,
                                                        uint32_t *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < 8 ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) s_warp[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  const uint32_t before = w > 0 ? s_warp[w - 1] : 0u;
  *total = s_warp[7];
  __syncthreads();
  return before + x - v;
}

// Decoupled look-back: sums the values of partitions part-1, part-2, ... until an inclusive
// entry is found, reading four predecessors per step so the walk costs a quarter of the L2
// round trips, and backing off while a predecessor has not published yet. Bounded: gives up
// (FGS_ERR_TIMEOUT) after `limit` empty polls, at once if limit = 0. The prefix it then
// returns is partial (smaller than the true one), so every offset built from it stays inside
// its buffer; the kernels after the scan see the status and do nothing.
__device__ __forceinline__ uint64_t look_back(const uint64_t *lb, int64_t part, int64_t stride,
                                              uint32_t *status, uint32_t limit) {
  uint64_t prefix = 0;
  uint32_t spins = 0;
  int64_t j = part - 1;
  if (limit == 0u && j >= 0) {
    set_status(status, ST_TIMEOUT);
    return 0;
  }
  while (j >= 0) {
    uint64_t st[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) st[q] = j - q >= 0 ? ld_volatile_u64(lb + (j - q) * stride) : LB_INC;
    int used = 0;
    bool done = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (done || used < q) break;
      const uint64_t flag = st[q] & ~LB_VAL;
      if (flag == 0) break;
      prefix += st[q] & LB_VAL;
      ++used;
      if (flag == LB_INC) done = true;
    }
    if (done) break;
    if (used == 0) {
      if (++spins > limit) {
        set_status(status, ST_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
    j -= used;
  }
  return prefix;
}

// Rect binning's tile counts without a pass over the pairs. A record's pairs are the first
// k = min(tiles_touched, w h) tiles of its w x h rect in row-major order (exactly what the pair
// walk emits): fr = k / w full rows and a partial row of k - fr w tiles. Each such block adds
// +1, -1, -1, +1 at the corners (x_lo, y_lo), (x_hi + 1, y_lo), (x_lo, y_hi + 1),
// (x_hi + 1, y_hi + 1) of a 2D difference grid held in tile_ranges[2t] (corners past the
// grid's edge are dropped: they only reach tiles beyond it); inclusive prefix sums along the
// rows and then the columns of every view (grid_scan_kernel) turn it into the per-tile pair
// counts. Eight atomics per record at most, instead of one per pair. A rect outside its view's
// grid (a malformed caller record) adds nothing, as the pair walk skips it.
__device__ __forceinline__ void rect_difference(const fgs_record *__restrict__ rec, uint32_t r,
                                                uint32_t tt_r, int64_t n_per_view,
                                                const Views &vs, uint32_t *ranges) {
  const uint4 w2 = __ldg(reinterpret_cast<const uint4 *>(rec + r) + 2);
  const uint32_t x0 = w2.z & 0xffffu, y0 = w2.z >> 16, x1 = w2.w & 0xffffu, y1 = w2.w >> 16;
  const View &V = vs.v[(int)(r / (uint32_t)n_per_view)];
  const uint32_t tiles_x = (uint32_t)V.tiles_x, tiles_y = (uint32_t)V.tiles_y;
  if (!(x0 <= x1 && y0 <= y1 && x1 < tiles_x && y1 < tiles_y)) return;
  const uint32_t w = x1 - x0 + 1u, h = y1 - y0 + 1u;
  const uint32_t k = (uint32_t)min((uint64_t)tt_r, (uint64_t)w * h);
  const uint32_t fr = k / w, rem = k - fr * w;
  uint32_t *grid = ranges + 2 * V.tile_offset;
  auto add = [&](uint32_t x, uint32_t y, uint32_t d) {
    if (x < tiles_x && y < tiles_y) atomicAdd(grid + 2 * ((size_t)y * tiles_x + x), d);
  };
  if (fr > 0u) {
    add(x0, y0, 1u); add(x1 + 1u, y0, 0xffffffffu);
    add(x0, y0 + fr, 0xffffffffu); add(x1 + 1u, y0 + fr, 1u);
  }
  if (rem > 0u) {
    const uint32_t y = y0 + fr;
    add(x0, y, 1u); add(x0 + rem, y, 0xffffffffu);
    add(x0, y + 1u, 0xffffffffu); add(x0 + rem, y + 1u, 1u);
  }
}

// The record scan. DIFF = true (rect binning) also adds every visible record to the tile-count
// difference grid (rect_difference) while its partition waits on the look-back; with more
// candidates than capacity the counts are then not used (the tile scan reads them as zero).
template <bool DIFF>
__global__ void __launch_bounds__(EMIT_THREADS)
    scan_kernel(const uint32_t *__restrict__ tt, int64_t R, int64_t capacity, int64_t *n_int,
                unsigned long long *n_cand, unsigned long long *n_vis, uint64_t *lb_pairs,
                uint64_t *lb_vis,
                uint32_t *part_counter, uint32_t *__restrict__ vis_rec,
                uint64_t *__restrict__ vis_off, uint32_t *__restrict__ chunk_first,
                uint32_t *status, uint32_t wait_limit, const fgs_record *__restrict__ rec,
                int64_t n_per_view, Views vs, uint32_t *ranges) {
  __shared__ uint32_t s_warp[8];
  __shared__ uint64_t s_prefix[2];
  __shared__ uint32_t s_part;
  const int tid = threadIdx.x;
  if (tid == 0) s_part = atomicAdd(part_counter, 1u);
  __syncthreads();
  const int64_t part = s_part;
  const int64_t base = part * EMIT_PART;
  if (FGS_CHECK && part == 0 && tid == 0) {  // the rasterizers' index bounds (checked build)
    WsHeader *h = reinterpret_cast<WsHeader *>(status);
    h->bounds_records = (uint32_t)R;
    h->bounds_pairs = (uint32_t)capacity;
    h->bounds_magic = BOUNDS_MAGIC;
  }

  uint32_t c[EMIT_ITEMS];
  uint32_t sum = 0, nv = 0;
#pragma unroll
  for (int k = 0; k < EMIT_ITEMS; ++k) {
    const int64_t r = base + tid * EMIT_ITEMS + k;
    c[k] = r < R ? tt[r] : 0u;
    sum += c[k];
    nv += c[k] > 0u ? 1u : 0u;
  }
  if (DIFF) {
#pragma unroll 4
    for (int k = 0; k < EMIT_ITEMS; ++k)
      if (c[k] > 0u)
        rect_difference(rec, (uint32_t)(base + tid * EMIT_ITEMS + k), c[k], n_per_view, vs, ranges);
  }
  uint32_t cta_pairs, cta_vis;
  uint32_t off = block_excl_scan_256(sum, s_warp, &cta_pairs);
  uint32_t voff = block_excl_scan_256(nv, s_warp, &cta_vis);
  // two look-backs at once: warp 0 for the pair offsets, warp 1 for the compacted ranks
  if ((tid & 31) == 0 && tid < 64) {
    uint64_t *lb = tid == 0 ? lb_pairs : lb_vis;
    const uint64_t agg = tid == 0 ? cta_pairs : cta_vis;
    uint64_t prefix = 0;
    if (part == 0) {
      st_volatile_u64(lb, LB_INC | agg);
    } else {
      st_volatile_u64(lb + part, LB_AGG | agg);
      prefix = look_back(lb, part, 1, status, wait_limit);
      st_volatile_u64(lb + part, LB_INC | (prefix + agg));
    }
    s_prefix[tid == 0 ? 0 : 1] = prefix;
    if (base + EMIT_PART >= R) {
      if (tid == 0) {
        *n_int = (int64_t)(prefix + agg);
        *n_cand = prefix + agg;
      } else {
        *n_vis = prefix + agg;
      }
    }
  }
  __syncthreads();
  const uint64_t pbase = s_prefix[0], vbase = s_prefix[1];
  uint64_t o = pbase + off;
  uint64_t v = vbase + voff;
#pragma unroll
  for (int k = 0; k < EMIT_ITEMS; ++k) {
    if (c[k] > 0u && in_bounds(v, (uint64_t)R, status)) {
      vis_rec[v] = (uint32_t)(base + tid * EMIT_ITEMS + k);
      vis_off[v] = o;
      // chunks whose first pair falls inside this record's pairs [o, o + c)
      const uint64_t end = min(o + c[k], (uint64_t)capacity);
      for (uint64_t ck = (o + EMIT_CHUNK - 1) / EMIT_CHUNK; ck * EMIT_CHUNK < end; ++ck)
        chunk_first[ck] = (uint32_t)v;
      ++v;
    }
    o += c[k];
  }
}

}  // namespace
}  // namespace fgs
