// scan.cuh - the block scan and the bounded decoupled look-back shared by the bin/sort kernels
// (binsort.cu, onesweep.cu), and the device-wide sort's record scan: a single-pass scan of
// tiles_touched with decoupled look-back. Included inside each file's anonymous namespace.
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

// The record scan of the device-wide sort: pair offsets of the records (decoupled look-back),
// the compacted list of records with pairs and the first record of every EMIT_CHUNK-pair chunk.
__global__ void __launch_bounds__(EMIT_THREADS)
    scan_kernel(const uint32_t *__restrict__ tt, int64_t R, int64_t capacity, int64_t *n_int,
                unsigned long long *n_cand, unsigned long long *n_vis, uint64_t *lb_pairs,
                uint64_t *lb_vis,
                uint32_t *part_counter, uint32_t *__restrict__ vis_rec,
                uint64_t *__restrict__ vis_off, uint32_t *__restrict__ chunk_first,
                uint32_t *status, uint32_t wait_limit) {
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
