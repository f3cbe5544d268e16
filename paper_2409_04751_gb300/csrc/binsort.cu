// binsort.cu - tile binning and key sort (Sec. 3.1 "Rendering"; Sec. 4.1 duplicateWithKeys and
// radixSort), sm_103a.
//
// The result is the one the method defines: for every (record, tile) pair of a record's tile
// rect, key = tile << 32 | depth bits and value = record, stably sorted by key, and each tile's
// [start, end) in the sorted arrays. Instead of a device-wide radix sort over all key bits
// (kept in onesweep.cu as the option FGS_BIN_ONESWEEP), the pairs are bucketed by tile first and
// each tile's bucket is sorted on its own:
//
//  1. scan_kernel: single-pass scan of tiles_touched with decoupled look-back (partitions of
//     4096 records claimed in order through an atomic counter). For every record with pairs it
//     writes its pair offset and its rank among such records (a compacted list), and for every
//     1024-pair chunk the rank of the record holding the chunk's first pair. For rect binning
//     it also adds each visible record to a 2D difference grid of tile counts (at most eight
//     atomics per record, rect_difference in scan.cuh).
//  2. rect binning: grid_scan_kernel turns the difference grid into the pairs of every tile
//     (row sums, then column sums). Exact (ellipse) binning: pair_kernel<false>, one CTA per
//     1024-pair chunk (the work per CTA is fixed however many tiles one Gaussian covers), counts
//     them pair by pair.
//  3. tile_scan_kernel: exclusive scan of the tile counts (decoupled look-back) gives every
//     tile's start; tiles are listed by segment size.
//  4. pair_kernel<true>: the same walk over the pairs claims a slot in the pair's tile bucket and
//     writes depth bits << 32 | record there.
//  5. segsort_kernel (one launch per size class): each tile's bucket is sorted in shared memory
//     (a one-pass bucket sort on the depth bits, or LSD radix passes when the depths are too
//     clustered for it) and written out as keys and values.
// Moving 8-byte words through memory twice (bucket write, bucket read) replaces the five to
// seven passes of a device-wide radix sort over (tile, depth) keys. The number of valid pairs
// is read on the device, so nothing here needs a host sync.
#include "fgs_internal.cuh"
#include "scan.cuh"

namespace fgs {

namespace {

// The (record, tile) pairs of one EMIT_CHUNK-pair chunk per CTA iteration, in pair order.
// The CTA loads the few records its chunk spans into shared memory and marks the first pair of
// each; a max-scan over the chunk then gives every pair its record. SCATTER = false: count the
// pairs of every tile (tile_ranges[2t]). SCATTER = true: claim a slot in the tile's bucket
// (tile_ranges[2t + 1] holds the bucket's next free slot) and write the word
// depth_bits << 32 | record there. Both passes visit the same pairs in the same way, so every
// bucket is filled exactly. Pairs whose tile falls outside their view's grid (a malformed
// caller record) are skipped by both.
template <bool SCATTER, bool ELLIPSE>
__global__ void __launch_bounds__(EMIT_THREADS)
    pair_kernel(const fgs_record *__restrict__ rec, int64_t n_per_view, Views vs,
                const uint32_t *__restrict__ vis_rec, const uint64_t *__restrict__ vis_off,
                const uint32_t *__restrict__ chunk_first, const unsigned long long *n_cand,
                const unsigned long long *n_vis, uint32_t *ranges, uint64_t *__restrict__ words,
                int64_t capacity, uint32_t *status) {
  constexpr int PER = EMIT_CHUNK / EMIT_THREADS;  // pairs per thread and chunk
  __shared__ uint32_t s_off[EMIT_CHUNK + 1];   // first pair of the record (clamped to hi)
  __shared__ uint32_t s_base[EMIT_CHUNK + 1];  // global tile id of the rect's corner (x0, y0)
  __shared__ uint32_t s_geom[EMIT_CHUNK + 1];  // rect width | rect height << 16 (0: skip)
  __shared__ uint32_t s_tx[EMIT_CHUNK + 1];    // the view's tiles_x
  __shared__ uint32_t s_depth[EMIT_CHUNK + 1];
  __shared__ uint32_t s_rec[EMIT_CHUNK + 1];
  __shared__ uint16_t s_own[EMIT_CHUNK];       // record (window slot) owning each pair
  __shared__ uint32_t s_wmax[EMIT_THREADS / 32];
  // exact mode: mean, conic, q* and the rect corner of each record of the window
  __shared__ float2 s_mu[ELLIPSE ? EMIT_CHUNK + 1 : 1];
  __shared__ float4 s_con[ELLIPSE ? EMIT_CHUNK + 1 : 1];
  __shared__ uint32_t s_rc[ELLIPSE ? EMIT_CHUNK + 1 : 1];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (binning_timed_out(status)) return;
  const int64_t total = (int64_t)*n_cand;
  if (!SCATTER && blockIdx.x == 0 && tid == 0 && total > capacity) set_status(status, ST_CAPACITY);
  const int64_t n = min(total, capacity);
  const int64_t nchunks = (n + EMIT_CHUNK - 1) / EMIT_CHUNK;
  const int64_t nv = (int64_t)*n_vis;

  for (int64_t ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const int64_t lo = ck * EMIT_CHUNK;
    const int64_t hi = min(lo + (int64_t)EMIT_CHUNK, n);
    const int64_t v0 = chunk_first[ck];
    const int64_t v1 = ck + 1 < nchunks ? (int64_t)chunk_first[ck + 1] : nv - 1;
    // records spanned by the chunk: the owner of pair lo and at most EMIT_CHUNK more (the
    // last chunk of a capacity-truncated emission may list more; they own no pair below hi)
    const int nw = (int)min(v1 - v0 + 1, (int64_t)EMIT_CHUNK + 1);
    // checked build: the chunk's records must lie in the compacted list (uniform per CTA)
    if (FGS_CHECK && (v1 < v0 || !in_bounds((uint64_t)(v0 + nw - 1), (uint64_t)nv, status))) {
      set_status(status, ST_BOUNDS);
      continue;
    }
    __syncthreads();
    for (int i = tid; i < EMIT_CHUNK; i += EMIT_THREADS) s_own[i] = 0;
    __syncthreads();
    for (int i = tid; i < nw; i += EMIT_THREADS) {
      uint32_t r = vis_rec[v0 + i];
      if (!in_bounds(r, (uint64_t)n_per_view * vs.n, status)) r = 0u;
      const uint4 w2 = __ldg(reinterpret_cast<const uint4 *>(rec + r) + 2);
      const uint32_t x0 = w2.z & 0xffffu, y0 = w2.z >> 16, x1 = w2.w & 0xffffu, y1 = w2.w >> 16;
      const int v = (int)(r / (uint32_t)n_per_view);
      const uint32_t tiles_x = (uint32_t)vs.v[v].tiles_x, tiles_y = (uint32_t)vs.v[v].tiles_y;
      const bool ok = x0 <= x1 && y0 <= y1 && x1 < tiles_x && y1 < tiles_y;
      const uint64_t off = vis_off[v0 + i];
      s_off[i] = (uint32_t)min(off, (uint64_t)hi);
      s_rec[i] = r;
      s_base[i] = (uint32_t)vs.v[v].tile_offset + y0 * tiles_x + x0;
      s_geom[i] = ok ? (x1 - x0 + 1u) | ((y1 - y0 + 1u) << 16) : 0u;
      s_tx[i] = tiles_x;
      s_depth[i] = w2.y;
      if (ELLIPSE) {
        const float4 w0 = __ldg(reinterpret_cast<const float4 *>(rec + r));
        const float4 w1 = __ldg(reinterpret_cast<const float4 *>(rec + r) + 1);
        s_mu[i] = make_float2(w0.x, w0.y);
        s_con[i] = make_float4(w0.z, w0.w, w1.x, fmaxf(2.f * logf(255.f * w1.y), 0.f));
        s_rc[i] = x0 | (y0 << 16);
      }
      if (i > 0 && off < (uint64_t)hi) s_own[off - (uint64_t)lo] = (uint16_t)i;
    }
    __syncthreads();
    // inclusive max-scan of the marks: thread t owns slots [PER t, PER t + PER)
    {
      uint32_t m[PER];
      uint32_t run = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        run = max(run, (uint32_t)s_own[tid * PER + k]);
        m[k] = run;
      }
      uint32_t x = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) x = max(x, __shfl_up_sync(0xffffffffu, x, o) * (lane >= o));
      if (lane == 31) s_wmax[wid] = x;
      uint32_t before = __shfl_up_sync(0xffffffffu, x, 1) * (lane >= 1);
      __syncthreads();
      for (int ww = 0; ww < wid; ++ww) before = max(before, s_wmax[ww]);
#pragma unroll
      for (int k = 0; k < PER; ++k) s_own[tid * PER + k] = (uint16_t)max(m[k], before);
    }
    __syncthreads();
    // each thread takes pairs tid, tid + 256, ... of the chunk: all their tiles first, then
    // all their atomics, so that a thread has several atomics in flight
    uint32_t tile[PER], owner[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int64_t j = lo + tid + k * EMIT_THREADS;
      tile[k] = 0xffffffffu;
      owner[k] = 0u;
      if (j < hi) {
        const uint32_t a = s_own[j - lo];
        const uint32_t geom = s_geom[a];
        const uint32_t local = (uint32_t)(j - lo) + (uint32_t)lo - s_off[a];
        const uint32_t w = geom & 0xffffu, h = geom >> 16;
        if (w != 0u) {
          // row inside the rect: float quotient (local < 2^22 is exact in FP32), corrected by one
          uint32_t dy = (uint32_t)((float)local * rcp_approx((float)w));
          if (dy * w > local) --dy;
          if ((dy + 1u) * w <= local) ++dy;
          const uint32_t dx = local - dy * w;
          // more pairs than the rect holds (a malformed record): skipped
          bool keep = dy < h && dx < w;
          if (ELLIPSE && keep) {
            const float2 mu = s_mu[a];
            const float4 cq = s_con[a];
            const uint32_t rc = s_rc[a];
            const float xl = (float)(((rc & 0xffffu) + dx) * TILE) + 0.5f;
            const float yl = (float)(((rc >> 16) + dy) * TILE) + 0.5f;
            keep = ellipse_reaches_tile(mu.x, mu.y, cq.x, cq.y, cq.z, cq.w, xl, xl + (TILE - 1),
                                        yl, yl + (TILE - 1));
          }
          if (keep) tile[k] = s_base[a] + dy * s_tx[a] + dx;
        }
        owner[k] = a;
      }
    }
    if (!SCATTER) {
#pragma unroll
      for (int k = 0; k < PER; ++k)
        if (tile[k] != 0xffffffffu) atomicAdd(&ranges[2 * (size_t)tile[k]], 1u);
    } else {
      uint32_t pos[PER];
#pragma unroll
      for (int k = 0; k < PER; ++k)
        pos[k] = tile[k] != 0xffffffffu ? atomicAdd(&ranges[2 * (size_t)tile[k] + 1], 1u) : 0xffffffffu;
      // checked build: with complete counts every claimed slot lies below the capacity
      if (FGS_CHECK && total <= capacity) {
#pragma unroll
        for (int k = 0; k < PER; ++k)
          if (tile[k] != 0xffffffffu) in_bounds(pos[k], (uint64_t)capacity, status);
      }
#pragma unroll
      for (int k = 0; k < PER; ++k)
        if (tile[k] != 0xffffffffu && (int64_t)pos[k] < capacity)
          words[pos[k]] = ((uint64_t)s_depth[owner[k]] << 32) | (uint64_t)s_rec[owner[k]];
    }
  }
}

// In-place inclusive prefix sums of the difference grid, one warp per line: ROWS = true sums
// along every view's tile rows, false along its columns (run after the rows). Sums are
// modulo 2^32, so the negative differences need no sign.
template <bool ROWS>
__global__ void __launch_bounds__(256)
    grid_scan_kernel(Views vs, int64_t n_lines, uint32_t *ranges,
                     const unsigned long long *n_cand, int64_t capacity,
                     const uint32_t *status) {
  if ((int64_t)*n_cand > capacity || binning_timed_out(status)) return;
  const int lane = threadIdx.x & 31;
  int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (g >= n_lines) return;
  int v = 0;
  for (; v < vs.n - 1; ++v) {
    const int64_t lines = ROWS ? vs.v[v].tiles_y : vs.v[v].tiles_x;
    if (g < lines) break;
    g -= lines;
  }
  const View &V = vs.v[v];
  const int64_t len = ROWS ? V.tiles_x : V.tiles_y;
  const int64_t step = ROWS ? 2 : 2 * (int64_t)V.tiles_x;  // words between consecutive entries
  uint32_t *p = ranges + 2 * (V.tile_offset + (ROWS ? g * V.tiles_x : g));
  uint32_t carry = 0u;
  for (int64_t c = 0; c < len; c += 32) {
    const int64_t j = c + lane;
    uint32_t x = j < len ? p[j * step] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    x += carry;
    if (j < len) p[j * step] = x;
    carry = __shfl_sync(0xffffffffu, x, 31);
  }
}

// Exclusive scan of the per-tile pair counts (tile_ranges[2t], written by the counting pass)
// over all tiles in global tile order, with decoupled look-back over partitions of TSCAN_PART
// tiles. Writes tile_ranges[t] = (start, start) for every non-empty tile (the second word is
// the scatter's cursor and ends as the tile's end) and appends the tile to the list of its
// segment-size class; empty tiles keep (0, 0). It runs even after the record scan gave up (its
// counts are then all zero), so that every partition publishes and no wait of its own look-back
// depends on a partition that left early.
__global__ void __launch_bounds__(256)
    tile_scan_kernel(uint32_t *ranges, int64_t total_tiles, uint64_t *lb,
                     uint32_t *part_counter, uint32_t *lists, uint32_t *seg_count,
                     const unsigned long long *n_cand, int64_t capacity, int64_t *n_int,
                     uint32_t *status, uint32_t wait_limit) {
  __shared__ uint32_t s_warp[8];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t s_part;
  __shared__ uint32_t s_cls[2], s_cls_base[2];
  const int tid = threadIdx.x;
  if (tid == 0) s_part = atomicAdd(part_counter, 1u);
  if (tid < 2) s_cls[tid] = 0u;
  __syncthreads();
  const int64_t part = s_part;
  const int64_t base = part * TSCAN_PART;
  // with more candidates than capacity the counts are not complete: read them as zero, and
  // report the overflow (the caller grows the buffers from the candidate count)
  const bool counts_ok = (int64_t)*n_cand <= capacity;
  if (!counts_ok && part == 0 && tid == 0) set_status(status, ST_CAPACITY);
  constexpr int ITEMS = TSCAN_PART / 256;
  uint32_t c[ITEMS];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int64_t t = base + tid * ITEMS + k;
    c[k] = t < total_tiles && counts_ok ? ranges[2 * t] : 0u;
    sum += c[k];
  }
  uint32_t agg;
  const uint32_t off = block_excl_scan_256(sum, s_warp, &agg);
  if (tid == 0) {
    uint64_t prefix = 0;
    if (part == 0) {
      st_volatile_u64(lb, LB_INC | agg);
    } else {
      st_volatile_u64(lb + part, LB_AGG | agg);
      prefix = look_back(lb, part, 1, status, wait_limit);
      st_volatile_u64(lb + part, LB_INC | (prefix + agg));
    }
    s_prefix = prefix;
    // the pairs kept (fewer than the candidates in the exact mode); with more candidates than
    // capacity the candidate count stays, so the caller can grow the buffers
    if (base + TSCAN_PART >= total_tiles && (int64_t)*n_cand <= capacity)
      *n_int = (int64_t)(prefix + agg);
  }
  // class ranks inside the CTA (order within a class list is irrelevant)
  uint32_t cls_rank[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int cls = c[k] <= (uint32_t)SEG_CAP0 ? 0 : 1;
    cls_rank[k] = c[k] > 0u ? atomicAdd(&s_cls[cls], 1u) : 0u;
  }
  __syncthreads();
  if (tid < 2) s_cls_base[tid] = s_cls[tid] ? atomicAdd(&seg_count[tid], s_cls[tid]) : 0u;
  __syncthreads();
  uint64_t o = s_prefix + off;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int64_t t = base + tid * ITEMS + k;
    if (c[k] > 0u) {
      ranges[2 * t] = (uint32_t)o;
      ranges[2 * t + 1] = (uint32_t)o;
      const int cls = c[k] <= (uint32_t)SEG_CAP0 ? 0 : 1;
      lists[(size_t)cls * (size_t)total_tiles + s_cls_base[cls] + cls_rank[k]] = (uint32_t)t;
    }
    o += c[k];
  }
}

// ------------------------------------------------------------------------------------------
// Per-tile segment sort. A tile's bucket holds its words depth_bits << 32 | record in
// arbitrary order; sorting the words as 64-bit integers orders them by depth and breaks depth
// ties by record index, which is the order a stable sort of the keys (tile << 32 | depth) in
// emission order gives. LSD radix passes over 8-bit digits, skipping digits that are equal in
// every word of the segment. A first attempt sorts the depth digits only; only a segment that
// then shows two equal depths is sorted again over all digits.
//
// Ranking is stable: warp w owns items [w * 32 * IPT, (w + 1) * 32 * IPT), taken 32 at a time
// in order; each group of 32 is ranked by warp multi-split (the lanes sharing a digit found
// through a per-warp shared bitmap that each lane ORs its bit into), and a per-warp digit
// counter carries the count over the groups.
template <int NT, int CAP>
struct SegSmem {
  uint64_t buf[CAP];
  union {
    struct {
      uint32_t wcnt[NT / 32][256];   // per-warp digit counts -> per-warp offsets within a digit
      uint32_t wmask[NT / 32][256];  // per-warp lane masks of one group of 32 (zero between groups)
    } rx;
    uint32_t cnt[CAP];               // bucket sort: sub-bucket counts -> starts
  };
  uint32_t dstart[256];         // digit start (exclusive prefix of the digit counts)
  uint32_t hist[256];           // chunked path: digit start over the whole segment
  uint32_t running[256];        // chunked path: digit count of the chunks already placed
  uint32_t wtot[NT / 32];
  uint64_t red[2][NT / 32];
};

template <int NT, int IPT, int CAP>
__device__ __forceinline__ void rank_items(SegSmem<NT, CAP> &S, const uint64_t (&x)[IPT],
                                           uint32_t cnt, int shift, uint32_t (&rank)[IPT]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = lane; e < 256; e += 32) S.rx.wcnt[w][e] = 0u;
  __syncwarp();
  if ((uint32_t)(w * 32 * IPT) < cnt) {
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
      const bool valid = li < cnt;
      const uint32_t d = (uint32_t)(x[k] >> shift) & 255u;
      // lanes holding the same digit: every lane sets its bit in the digit's mask
      if (valid) atomicOr(&S.rx.wmask[w][d], 1u << lane);
      __syncwarp();
      const uint32_t peers = valid ? S.rx.wmask[w][d] : 0u;
      const uint32_t before = __popc(peers & lt);
      uint32_t c = 0;
      if (valid) c = S.rx.wcnt[w][d];
      __syncwarp();
      if (valid && before == 0u) {
        S.rx.wcnt[w][d] = c + __popc(peers);
        S.rx.wmask[w][d] = 0u;
      }
      __syncwarp();
      rank[k] = c + before;
    }
  }
  __syncthreads();
}

// Turns S.rx.wcnt[w][d] (counts) into per-warp exclusive offsets within digit d and S.dstart[d]
// into the exclusive prefix of the digit totals; returns digit tid's total (tid < 256).
template <int NT, int IPT, int CAP>
__device__ __forceinline__ uint32_t digit_offsets(SegSmem<NT, CAP> &S) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint32_t dcount = 0, incl = 0;
  if (tid < 256) {
#pragma unroll 4
    for (int ww = 0; ww < NT / 32; ++ww) {
      const uint32_t c = S.rx.wcnt[ww][tid];
      S.rx.wcnt[ww][tid] = dcount;
      dcount += c;
    }
    incl = dcount;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) S.wtot[w] = incl;
  }
  __syncthreads();
  if (tid < 256) {
    uint32_t before = 0;
    for (int ww = 0; ww < w; ++ww) before += S.wtot[ww];
    S.dstart[tid] = before + incl - dcount;
  }
  __syncthreads();
  return dcount;
}

// Block AND / OR of a 64-bit value; every thread gets the results.
template <int NT, int IPT, int CAP>
__device__ __forceinline__ void block_and_or(SegSmem<NT, CAP> &S, uint64_t &a, uint64_t &o) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    a &= __shfl_xor_sync(0xffffffffu, a, s);
    o |= __shfl_xor_sync(0xffffffffu, o, s);
  }
  if (lane == 0) {
    S.red[0][w] = a;
    S.red[1][w] = o;
  }
  __syncthreads();
  a = ~0ull;
  o = 0ull;
  for (int ww = 0; ww < NT / 32; ++ww) {
    a &= S.red[0][ww];
    o |= S.red[1][ww];
  }
  __syncthreads();
}

// One stable pass over the digit at `shift` of the segment held in registers (x) and shared
// memory; leaves the result in both.
template <int NT, int IPT, int CAP>
__device__ __forceinline__ void smem_pass(SegSmem<NT, CAP> &S, uint64_t (&x)[IPT], uint32_t cnt,
                                          int shift) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t rank[IPT];
  rank_items<NT, IPT, CAP>(S, x, cnt, shift, rank);
  digit_offsets<NT, IPT, CAP>(S);
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    if (li < cnt) {
      const uint32_t d = (uint32_t)(x[k] >> shift) & 255u;
      S.buf[S.dstart[d] + S.rx.wcnt[w][d] + rank[k]] = x[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    x[k] = li < cnt ? S.buf[li] : 0ull;
  }
}

// Sort one segment of cnt <= NT * IPT words in shared memory and write keys / values.
template <int NT, int IPT, int CAP>
__device__ __forceinline__ void sort_segment_smem(SegSmem<NT, CAP> &S, const uint64_t *src,
                                                  uint32_t cnt, uint64_t tile,
                                                  uint64_t *kout, uint32_t *vout) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // the lane masks share storage with the bucket sort's counters: clear them first
  for (int e = threadIdx.x; e < (NT / 32) * 256; e += NT) (&S.rx.wmask[0][0])[e] = 0u;
  __syncthreads();
  uint64_t x[IPT];
  uint64_t a = ~0ull, o = 0ull;
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    x[k] = li < cnt ? src[li] : 0ull;
    if (li < cnt) {
      S.buf[li] = x[k];
      a &= x[k];
      o |= x[k];
    }
  }
  block_and_or<NT, IPT, CAP>(S, a, o);
  const uint64_t varying = a ^ o;
#pragma unroll
  for (int p = 4; p < 8; ++p)
    if ((varying >> (8 * p)) & 255u) smem_pass<NT, IPT, CAP>(S, x, cnt, 8 * p);
  // equal depths (the high halves) in adjacent slots: sort again over every digit
  bool tie = false;
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    if (li + 1 < cnt) tie |= (S.buf[li] >> 32) == (S.buf[li + 1] >> 32);
  }
  if (__syncthreads_or(tie)) {
#pragma unroll
    for (int p = 0; p < 8; ++p)
      if ((varying >> (8 * p)) & 255u) smem_pass<NT, IPT, CAP>(S, x, cnt, 8 * p);
  }
  for (uint32_t i = threadIdx.x; i < cnt; i += NT) {
    const uint64_t v = S.buf[i];
    kout[i] = (tile << 32) | (v >> 32);
    vout[i] = (uint32_t)v;
  }
  __syncthreads();  // buf reused by the next segment
}

// Bucket sort of one segment of cnt <= NT * IPT words, the usual path. The depth bits of the
// segment span [kmin, kmax]; the words are counted into NB sub-buckets (NB = the power of two
// >= cnt, at least 32) by the leading bits of depth - kmin (one shared atomic per word, which
// also gives the word its slot), the counts are scanned, the words placed by sub-bucket, and each
// word's final place is its sub-bucket's start plus the number of smaller words in its
// sub-bucket. Words are distinct (the record index is in the low half), so this is a total order
// equal to that of the 64-bit words. Returns false, having written nothing, when a sub-bucket
// holds more than BUCKET_KMAX words (depths clustered tighter than the sub-bucket width, or many
// equal depths); the radix path then sorts the segment.
constexpr uint32_t BUCKET_KMAX = 32;

template <int NT, int IPT, int CAP>
__device__ __forceinline__ bool bucket_sort_segment(SegSmem<NT, CAP> &S, const uint64_t *src,
                                                    uint32_t cnt, uint64_t tile,
                                                    uint64_t *kout, uint32_t *vout) {
  static_assert(NT * IPT <= CAP, "capacity");
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // NB sub-buckets: CAP for the small class (fixed, so the counter loops unroll), else the
  // power of two >= cnt, so that a segment of the large class pays for its own length only
  constexpr bool FIXED = CAP <= SEG_CAP0;
  constexpr int LOGCAP = CAP == 1024 ? 10 : (CAP == 2048 ? 11 : (CAP == 4096 ? 12 : 13));
  static_assert((1 << LOGCAP) == CAP, "sub-bucket count");
  const int lognb = FIXED ? LOGCAP : max(5, 32 - __clz(cnt - 1u));
  const uint32_t nb = 1u << lognb;
  const uint32_t cpt = nb > (uint32_t)NT ? nb / NT : 1u;  // counters per thread in the scan
  uint64_t x[IPT];
  uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(k * NT + tid);
    x[k] = li < cnt ? src[li] : 0ull;
    if (li < cnt) {
      const uint32_t h = (uint32_t)(x[k] >> 32);
      kmin = min(kmin, h);
      kmax = max(kmax, h);
    }
  }
  if (FIXED) {
#pragma unroll
    for (int q = 0; q < CAP / NT; ++q) S.cnt[q * NT + tid] = 0u;
  } else {
    for (uint32_t q = tid; q < nb; q += NT) S.cnt[q] = 0u;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, s));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, s));
  }
  if (lane == 0) {
    S.red[0][w] = kmin;
    S.red[1][w] = kmax;
  }
  __syncthreads();
  kmin = 0xffffffffu;
  kmax = 0u;
  for (int ww = 0; ww < NT / 32; ++ww) {
    kmin = min(kmin, (uint32_t)S.red[0][ww]);
    kmax = max(kmax, (uint32_t)S.red[1][ww]);
  }
  const uint32_t span = kmax - kmin;
  const int bits = span ? 32 - __clz(span) : 0;
  const int sh = bits > lognb ? bits - lognb : 0;  // (depth - kmin) >> sh < NB
  // per word: sub-bucket << 18 | slot in the sub-bucket (a slot beyond BUCKET_KMAX is never
  // used: the segment then goes to the radix path)
  uint32_t bs[IPT];
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(k * NT + tid);
    bs[k] = 0u;
    if (li < cnt) {
      const uint32_t b = ((uint32_t)(x[k] >> 32) - kmin) >> sh;
      bs[k] = (b << 18) | min(atomicAdd(&S.cnt[b], 1u), 0x3ffffu);
    }
  }
  __syncthreads();
  // exclusive scan of the counts (thread tid owns counters [cpt tid, cpt tid + cpt) below NB)
  // and the largest count
  const uint32_t q0 = (uint32_t)tid * cpt;
  uint32_t tot = 0, mx = 0;
  if (FIXED) {
#pragma unroll
    for (int q = 0; q < CAP / NT; ++q) {
      const uint32_t v = S.cnt[q0 + q];
      tot += v;
      mx = max(mx, v);
    }
  } else if (q0 < nb) {
    for (uint32_t q = q0; q < q0 + cpt; ++q) {
      const uint32_t v = S.cnt[q];
      tot += v;
      mx = max(mx, v);
    }
  }
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, s));
  __syncthreads();  // everyone has read S.red
  if (lane == 31) S.wtot[w] = incl;
  if (lane == 0) S.red[0][w] = mx;
  __syncthreads();
  uint32_t before = 0;
  for (int ww = 0; ww < w; ++ww) before += S.wtot[ww];
  mx = 0;
  for (int ww = 0; ww < NT / 32; ++ww) mx = max(mx, (uint32_t)S.red[0][ww]);
  if (FIXED) {
    uint32_t e = before + incl - tot;
#pragma unroll
    for (int q = 0; q < CAP / NT; ++q) {
      const uint32_t v = S.cnt[q0 + q];
      S.cnt[q0 + q] = e;
      e += v;
    }
  } else if (q0 < nb) {
    uint32_t e = before + incl - tot;
    for (uint32_t q = q0; q < q0 + cpt; ++q) {
      const uint32_t v = S.cnt[q];
      S.cnt[q] = e;
      e += v;
    }
  }
  __syncthreads();
  if (mx > BUCKET_KMAX) return false;  // uniform over the CTA
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(k * NT + tid);
    if (li < cnt) S.buf[S.cnt[bs[k] >> 18] + (bs[k] & 0x3ffffu)] = x[k];
  }
  __syncthreads();
  // final place: start of the sub-bucket + number of smaller words in it (bs[k] becomes it)
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(k * NT + tid);
    if (li < cnt) {
      const uint32_t b = bs[k] >> 18;
      const uint32_t b0 = S.cnt[b];
      const uint32_t b1 = b + 1u < nb ? S.cnt[b + 1u] : cnt;
      uint32_t r = 0;
      for (uint32_t j = b0; j < b1; ++j) r += S.buf[j] < x[k] ? 1u : 0u;
      bs[k] = b0 + r;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(k * NT + tid);
    if (li < cnt) S.buf[bs[k]] = x[k];
  }
  __syncthreads();
  for (uint32_t i = tid; i < cnt; i += NT) {
    const uint64_t v = S.buf[i];
    kout[i] = (tile << 32) | (v >> 32);
    vout[i] = (uint32_t)v;
  }
  __syncthreads();  // buf and counters reused by the next segment
  return true;
}

// Sort one segment longer than NT * IPT through global memory: per digit, a histogram pass
// over the segment, then the segment in chunks of NT * IPT words in order, each ranked in
// shared memory and scattered to its place in the other buffer (words <-> the key output,
// which serves as scratch). All digits with varying bits are sorted. The last step turns the
// words into keys and values wherever the data ended (in place if that is the key output).
template <int NT, int IPT, int CAP>
__device__ __noinline__ void sort_segment_chunked(SegSmem<NT, CAP> &S, uint64_t *words, uint32_t cnt,
                                     uint64_t tile, uint64_t *kout, uint32_t *vout) {
  constexpr uint32_t CH = NT * IPT;  // words per chunk
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int e = tid; e < (NT / 32) * 256; e += NT) (&S.rx.wmask[0][0])[e] = 0u;
  uint64_t a = ~0ull, o = 0ull;
  for (uint32_t i = tid; i < cnt; i += NT) {
    const uint64_t v = words[i];
    a &= v;
    o |= v;
  }
  block_and_or<NT, IPT, CAP>(S, a, o);
  const uint64_t varying = a ^ o;
  uint64_t *src = words, *dst = kout;
  for (int p = 0; p < 8; ++p) {
    if (((varying >> (8 * p)) & 255u) == 0u) continue;
    const int shift = 8 * p;
    for (int e = tid; e < 256; e += NT) {
      S.hist[e] = 0u;
      S.running[e] = 0u;
    }
    __syncthreads();
    for (uint32_t i = tid; i < cnt; i += NT) atomicAdd(&S.hist[(uint32_t)(src[i] >> shift) & 255u], 1u);
    __syncthreads();
    {  // exclusive scan of the histogram in place
      uint32_t c = 0, incl = 0;
      if (tid < 256) {
        c = S.hist[tid];
        incl = c;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, s);
          if (lane >= s) incl += y;
        }
        if (lane == 31) S.wtot[w] = incl;
      }
      __syncthreads();
      if (tid < 256) {
        uint32_t before = 0;
        for (int ww = 0; ww < w; ++ww) before += S.wtot[ww];
        S.hist[tid] = before + incl - c;
      }
      __syncthreads();
    }
    for (uint32_t lo = 0; lo < cnt; lo += CH) {
      const uint32_t ccnt = min(CH, cnt - lo);
      uint64_t x[IPT];
      uint32_t rank[IPT];
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
        x[k] = li < ccnt ? src[lo + li] : 0ull;
      }
      rank_items<NT, IPT, CAP>(S, x, ccnt, shift, rank);
      const uint32_t dcount = digit_offsets<NT, IPT, CAP>(S);
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
        if (li < ccnt) {
          const uint32_t d = (uint32_t)(x[k] >> shift) & 255u;
          dst[S.hist[d] + S.running[d] + S.rx.wcnt[w][d] + rank[k]] = x[k];
        }
      }
      __syncthreads();
      if (tid < 256) S.running[tid] += dcount;
      __syncthreads();
    }
    uint64_t *t = src;
    src = dst;
    dst = t;
  }
  for (uint32_t i = tid; i < cnt; i += NT) {
    const uint64_t v = src[i];
    kout[i] = (tile << 32) | (v >> 32);
    vout[i] = (uint32_t)v;
  }
  __syncthreads();
}

// One CTA per listed tile of a size class, persistent over the class list.
// The radix path kept out of line for the large class, where inlining it would raise the
// register needs of the bucket sort that every segment takes first.
template <int NT, int IPT, int CAP>
__device__ __noinline__ void sort_segment_smem_outlined(SegSmem<NT, CAP> &S, const uint64_t *src,
                                                        uint32_t cnt, uint64_t tile,
                                                        uint64_t *kout, uint32_t *vout) {
  sort_segment_smem<NT, IPT, CAP>(S, src, cnt, tile, kout, vout);
}

// Sort one segment of cnt <= NT * IPT words in shared memory: the bucket sort, or the radix
// passes if the bucket sort declines.
template <int NT, int IPT, int CAP>
__device__ __forceinline__ void sort_segment(SegSmem<NT, CAP> &S, uint64_t *words, uint32_t cnt,
                                             uint64_t tile, uint64_t *kout, uint32_t *vout) {
  if (bucket_sort_segment<NT, IPT, CAP>(S, words, cnt, tile, kout, vout)) return;
  if constexpr (CAP <= SEG_CAP0)
    sort_segment_smem<NT, IPT, CAP>(S, words, cnt, tile, kout, vout);
  else
    sort_segment_smem_outlined<NT, IPT, CAP>(S, words, cnt, tile, kout, vout);
}

// One CTA per listed tile of a size class, persistent over the class list. The number of words
// per thread is picked per segment (the smallest of IPT_LO, 2 IPT_LO, ... that holds it), so a
// segment costs in proportion to its own length, not the class's largest.
template <int NT, int IPT_LO, int CAP, int MIN_BLOCKS, bool CHUNKED>
__global__ void __launch_bounds__(NT, MIN_BLOCKS)
    segsort_kernel(const uint32_t *__restrict__ list, const uint32_t *list_count,
                   const uint32_t *__restrict__ ranges, uint64_t *words, uint64_t *keys,
                   uint32_t *vals, int64_t capacity, int64_t total_tiles, uint32_t *status) {
  static_assert(NT * IPT_LO * 2 == CAP, "two word counts per class");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SegSmem<NT, CAP> &S = *reinterpret_cast<SegSmem<NT, CAP> *>(smem_raw);
  if (binning_timed_out(status)) return;
  uint32_t count = *list_count;
  if (!in_bounds(count, (uint64_t)total_tiles + 1u, status)) count = 0u;
  for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const uint32_t t = __ldg(list + i);
    if (!in_bounds(t, (uint64_t)total_tiles, status)) continue;
    const uint2 rg = __ldg(reinterpret_cast<const uint2 *>(ranges) + t);
    // bounds of a bucket that a device-side error left inconsistent: skip it (a listed tile is
    // never empty, so the checked build reports it)
    if (rg.y <= rg.x || (int64_t)rg.y > capacity) {
      if (FGS_CHECK) set_status(status, ST_BOUNDS);
      continue;
    }
    const uint32_t cnt = rg.y - rg.x;
    if (cnt <= (uint32_t)(NT * IPT_LO))
      sort_segment<NT, IPT_LO, CAP>(S, words + rg.x, cnt, t, keys + rg.x, vals + rg.x);
    else if (cnt <= (uint32_t)CAP)
      sort_segment<NT, 2 * IPT_LO, CAP>(S, words + rg.x, cnt, t, keys + rg.x, vals + rg.x);
    else if (CHUNKED)
      sort_segment_chunked<NT, 2 * IPT_LO, CAP>(S, words + rg.x, cnt, t, keys + rg.x, vals + rg.x);
    else if (FGS_CHECK)
      set_status(status, ST_BOUNDS);  // a long segment listed in the short class
  }
}

template <int NT, int IPT_LO, int CAP, int MIN_BLOCKS, bool CHUNKED>
cudaError_t launch_segsort(const uint32_t *list, const uint32_t *list_count,
                           const uint32_t *ranges, uint64_t *words, uint64_t *keys,
                           uint32_t *vals, int64_t capacity, int64_t total_tiles,
                           uint32_t *status, cudaStream_t st) {
  constexpr size_t smem = sizeof(SegSmem<NT, CAP>);
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaFuncSetAttribute(segsort_kernel<NT, IPT_LO, CAP, MIN_BLOCKS, CHUNKED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, segsort_kernel<NT, IPT_LO, CAP, MIN_BLOCKS, CHUNKED>, NT, smem);
    occ = a > 0 ? a : 1;
  }
  segsort_kernel<NT, IPT_LO, CAP, MIN_BLOCKS, CHUNKED><<<(unsigned)(sm_count() * occ), NT, smem, st>>>(
      list, list_count, ranges, words, keys, vals, capacity, total_tiles, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bin_sort(const fgs_record *records, const uint32_t *tiles_touched,
                            int64_t n, const Views &vs, uint64_t *keys, uint32_t *vals,
                            int64_t capacity, uint32_t *tile_ranges, int64_t *n_int,
                            char *ws, const WsLayout &L, uint32_t flags,
                            const CallOpts &opt, cudaStream_t st) {
  cudaError_t e;
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.header);
  uint64_t *scan_lb = reinterpret_cast<uint64_t *>(ws + L.scan_lb);
  uint64_t *tile_lb = reinterpret_cast<uint64_t *>(ws + L.tile_lb);
  uint32_t *lists = reinterpret_cast<uint32_t *>(ws + L.seg_list);
  uint64_t *words = reinterpret_cast<uint64_t *>(ws + L.words);
  uint32_t *vis_rec = reinterpret_cast<uint32_t *>(ws + L.vis_rec);
  uint64_t *vis_off = reinterpret_cast<uint64_t *>(ws + L.vis_off);
  uint32_t *chunk_first = reinterpret_cast<uint32_t *>(ws + L.chunk_first);
  const int64_t R = (int64_t)vs.n * n;
  const int64_t T = vs.total_tiles;

  // the header and both look-back arrays are adjacent: one memset
  if ((e = cudaMemsetAsync(hdr, 0, L.g2d - L.header, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)T, st)) != cudaSuccess) return e;
  if (R == 0) return cudaMemsetAsync(n_int, 0, sizeof(int64_t), st);

  const bool ellipse = (flags & FGS_BIN_ELLIPSE) != 0;
  // rect binning: the record scan also builds the tile-count difference grid
  if (ellipse)
    scan_kernel<false><<<(unsigned)L.scan_parts, EMIT_THREADS, 0, st>>>(
        tiles_touched, R, capacity, n_int, &hdr->n_candidates, &hdr->n_visible, scan_lb,
        scan_lb + L.scan_parts, &hdr->scan_parts, vis_rec, vis_off, chunk_first, &hdr->status,
        opt.wait_limit, records, n, vs, tile_ranges);
  else
    scan_kernel<true><<<(unsigned)L.scan_parts, EMIT_THREADS, 0, st>>>(
        tiles_touched, R, capacity, n_int, &hdr->n_candidates, &hdr->n_visible, scan_lb,
        scan_lb + L.scan_parts, &hdr->scan_parts, vis_rec, vis_off, chunk_first, &hdr->status,
        opt.wait_limit, records, n, vs, tile_ranges);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // two waves of the 8 CTAs an SM holds: the pair walks wait on record loads and returning
  // atomics, so more chunks in flight hide more of that latency
  int64_t egrid = (int64_t)sm_count() * 16;
  if (egrid > L.chunks) egrid = L.chunks;
  if (egrid < 1) egrid = 1;
  if (ellipse) {
    pair_kernel<false, true><<<(unsigned)egrid, EMIT_THREADS, 0, st>>>(
        records, n, vs, vis_rec, vis_off, chunk_first, &hdr->n_candidates, &hdr->n_visible,
        tile_ranges, words, capacity, &hdr->status);
  } else {
    int64_t rows = 0, cols = 0;
    for (int v = 0; v < vs.n; ++v) {
      rows += vs.v[v].tiles_y;
      cols += vs.v[v].tiles_x;
    }
    grid_scan_kernel<true><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(
        vs, rows, tile_ranges, &hdr->n_candidates, capacity, &hdr->status);
    grid_scan_kernel<false><<<(unsigned)((cols * 32 + 255) / 256), 256, 0, st>>>(
        vs, cols, tile_ranges, &hdr->n_candidates, capacity, &hdr->status);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tile_scan_kernel<<<(unsigned)L.tile_parts, 256, 0, st>>>(
      tile_ranges, T, tile_lb, &hdr->tile_parts, lists, hdr->seg_count, &hdr->n_candidates,
      capacity, n_int, &hdr->status, opt.wait_limit);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ellipse)
    pair_kernel<true, true><<<(unsigned)egrid, EMIT_THREADS, 0, st>>>(
        records, n, vs, vis_rec, vis_off, chunk_first, &hdr->n_candidates, &hdr->n_visible,
        tile_ranges, words, capacity, &hdr->status);
  else
    pair_kernel<true, false><<<(unsigned)egrid, EMIT_THREADS, 0, st>>>(
        records, n, vs, vis_rec, vis_off, chunk_first, &hdr->n_candidates, &hdr->n_visible,
        tile_ranges, words, capacity, &hdr->status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_segsort<256, 2, SEG_CAP0, 6, false>(lists, &hdr->seg_count[0], tile_ranges,
                                                       words, keys, vals, capacity, T,
                                                       &hdr->status, st)) != cudaSuccess)
    return e;
  return launch_segsort<512, 8, SEG_CAP1, 1, true>(lists + T, &hdr->seg_count[1], tile_ranges,
                                                   words, keys, vals, capacity, T,
                                                   &hdr->status, st);
}

}  // namespace fgs
