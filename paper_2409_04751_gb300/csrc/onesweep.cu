// onesweep.cu - the device-wide radix sort of the (tile, depth) keys (Sec. 3.1 "Rendering";
// Sec. 4.1 duplicateWithKeys and radixSort), sm_103a: the renderer's own sort design, kept as
// an option of fgs_bin_sort_ex (FGS_BIN_ONESWEEP) beside the tile-bucketed default of
// binsort.cu. Same output bit for bit.
//
//  1. scan_kernel (scan.cuh): pair offsets, compacted record list, chunk starts.
//  2. emit_kernel: one CTA per 1024-pair chunk (fixed work per CTA); each pair finds its record
//     by binary search in a shared-memory window and writes key = tile << 32 | depth bits,
//     value = record, coalesced. The same pass counts the 8-bit digit histograms of every radix
//     pass (warp-aggregated shared atomics), so the sort needs no separate histogram read.
//     A pair beyond its record's rect (tiles_touched larger than the rect's area, or a rect
//     outside its view's grid) gets the tile id total_tiles, one past the last tile: it sorts
//     after every kept pair, no tile range takes it, and it is not counted in the result, so
//     the output is the default sort's for such records too.
//  3. onesweep_kernel (one launch per 8-bit digit): Adinets & Merrill's single-pass LSD radix
//     sort: each partition of 4096 keys is ranked in shared memory (warp multi-split with
//     match_any, stable), publishes its per-digit counts, resolves its global digit offsets by
//     decoupled look-back over earlier partitions (bounded waits), and scatters through shared
//     memory so that runs of equal digits are written contiguously. Persistent cooperative CTAs
//     take partitions round-robin, TMA double-buffered. When (tile, depth, record) fit 64 bits
//     the passes move packed 8-byte words and the last pass unpacks them.
//  4. ranges_kernel: [start, end) of every tile in the sorted keys.
#include "fgs_internal.cuh"
#include "scan.cuh"

namespace fgs {

namespace {

__global__ void __launch_bounds__(EMIT_THREADS)
    emit_kernel(const fgs_record *__restrict__ rec, int64_t n_per_view, Views vs,
                const uint32_t *__restrict__ vis_rec, const uint64_t *__restrict__ vis_off,
                const uint32_t *__restrict__ chunk_first, const int64_t *n_int,
                const unsigned long long *n_vis, uint64_t *__restrict__ keys,
                uint32_t *__restrict__ vals, int64_t capacity, uint32_t *hist, int passes,
                int idx_bits, int packed, unsigned long long *n_dropped, uint32_t *status) {
  __shared__ uint64_t s_off[EMIT_CHUNK + 1];
  __shared__ uint32_t s_base[EMIT_CHUNK + 1];   // global tile id of the rect's corner (x0, y0)
  __shared__ uint32_t s_geom[EMIT_CHUNK + 1];   // rect width | view tiles_x << 16
  __shared__ uint32_t s_rows[EMIT_CHUNK + 1];   // rect height (0: a rect outside the grid)
  __shared__ uint32_t s_depth[EMIT_CHUNK + 1];
  __shared__ uint32_t s_rec[EMIT_CHUNK + 1];
  __shared__ uint32_t s_hist[SORT_MAX_PASSES * 256];
  __shared__ uint32_t s_drop;
  const int tid = threadIdx.x;
  if (binning_timed_out(status)) return;
  const uint32_t drop_tile = (uint32_t)vs.total_tiles;  // one past the last tile
  const int64_t total = *n_int;
  if (tid == 0 && total > capacity) set_status(status, ST_CAPACITY);
  const int64_t n = min(total, capacity);
  const int64_t nchunks = (n + EMIT_CHUNK - 1) / EMIT_CHUNK;
  const int64_t nv = (int64_t)*n_vis;
  for (int e = tid; e < passes * 256; e += EMIT_THREADS) s_hist[e] = 0u;
  if (tid == 0) s_drop = 0u;

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
    for (int i = tid; i < nw; i += EMIT_THREADS) {
      uint32_t r = vis_rec[v0 + i];
      if (!in_bounds(r, (uint64_t)n_per_view * vs.n, status)) r = 0u;
      const uint4 w2 = __ldg(reinterpret_cast<const uint4 *>(rec + r) + 2);
      const uint32_t x0 = w2.z & 0xffffu, y0 = w2.z >> 16, x1 = w2.w & 0xffffu, y1 = w2.w >> 16;
      const int v = (int)(r / (uint32_t)n_per_view);
      const uint32_t tiles_x = (uint32_t)vs.v[v].tiles_x, tiles_y = (uint32_t)vs.v[v].tiles_y;
      const bool ok = x0 <= x1 && y0 <= y1 && x1 < tiles_x && y1 < tiles_y;
      s_off[i] = vis_off[v0 + i];
      s_rec[i] = r;
      s_base[i] = (uint32_t)vs.v[v].tile_offset + y0 * tiles_x + x0;
      s_geom[i] = (ok ? x1 - x0 + 1u : 1u) | (tiles_x << 16);
      s_rows[i] = ok ? y1 - y0 + 1u : 0u;
      s_depth[i] = w2.y;
    }
    __syncthreads();
    // depth digits (passes 0-3) are the same for all pairs of a record: count them once per
    // record with the number of its pairs inside this chunk
    for (int i = tid; i < nw; i += EMIT_THREADS) {
      const uint64_t a0 = s_off[i] > (uint64_t)lo ? s_off[i] : (uint64_t)lo;
      const uint64_t a1 = i + 1 < nw ? (s_off[i + 1] < (uint64_t)hi ? s_off[i + 1] : (uint64_t)hi)
                                     : (uint64_t)hi;
      if (a1 > a0) {
        const uint32_t cnt = (uint32_t)(a1 - a0), dep = s_depth[i];
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p * 256 + ((dep >> (8 * p)) & 255u)], cnt);
      }
    }
    for (int64_t jb = lo; jb < hi; jb += EMIT_THREADS) {
      const int64_t j = jb + tid;
      const bool valid = j < hi;
      uint64_t key = 0;
      if (valid) {
        int a = 0, b = nw;  // s_off[a] <= j < s_off[b] (s_off[nw] taken as +inf)
        while (b - a > 1) {
          const int mid = (a + b) >> 1;
          if (s_off[mid] <= (uint64_t)j) a = mid; else b = mid;
        }
        const uint32_t local = (uint32_t)((uint64_t)j - s_off[a]);
        const uint32_t geom = s_geom[a];
        const uint32_t w = geom & 0xffffu, tiles_x = geom >> 16;
        // row inside the rect: float quotient (local < 2^22 is exact in FP32) corrected by one
        uint32_t dy = (uint32_t)((float)local * rcp_approx((float)w));
        if (dy * w > local) --dy;
        if ((dy + 1u) * w <= local) ++dy;
        const bool kept = dy < s_rows[a];
        const uint32_t tile = kept ? s_base[a] + dy * tiles_x + (local - dy * w) : drop_tile;
        if (!kept) atomicAdd(&s_drop, 1u);
        key = ((uint64_t)tile << 32) | (uint64_t)s_depth[a];
        if (packed) {
          keys[j] = (key << idx_bits) | (uint64_t)s_rec[a];
        } else {
          keys[j] = key;
          vals[j] = s_rec[a];
        }
      }
      // tile digits: the lowest changes from pair to pair along a rect row (plain atomics
      // rarely collide); higher ones are shared by runs of pairs (warp-aggregated)
      if (passes > 4 && valid) atomicAdd(&s_hist[4 * 256 + ((uint32_t)(key >> 32) & 255u)], 1u);
      for (int p = 5; p < passes; ++p) {
        const uint32_t d = valid ? (uint32_t)(key >> (8 * p)) & 255u : 0x100u + (threadIdx.x & 31);
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lanemask_lt()) == 0u) atomicAdd(&s_hist[p * 256 + d], __popc(peers));
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < passes * 256; e += EMIT_THREADS)
    if (s_hist[e]) atomicAdd(hist + e, s_hist[e]);
  if (tid == 0 && s_drop) atomicAdd(n_dropped, (unsigned long long)s_drop);
}

// Shared memory of one onesweep CTA: two input buffers filled by TMA bulk copies (the next
// partition lands in one while the current one is ranked in the other, which then serves as
// the exchange buffer of the local scatter), per-warp digit counters and digit offsets.
template <bool KV>
struct SortSmem {
  uint64_t keys[2][SORT_PART];
  uint32_t vals[KV ? 2 : 1][KV ? SORT_PART : 4];
  uint32_t wcnt[SORT_THREADS / 32][256];  // per-warp digit counts -> per-warp offsets
  uint32_t local_start[256];               // digit start inside the partition
  uint32_t global_base[256];               // digit base in the output for this partition
  uint32_t hist_excl[256];                 // exclusive scan of this pass's global histogram
  uint32_t warp_tmp[8];
  uint32_t part[2];
  uint64_t bar[2];
};

// Issue the TMA bulk copies of partition `part` into buffer `b`: the 16-byte-aligned prefix
// of its keys (and values); the few trailing elements of a ragged last partition are loaded
// with plain loads after the wait.
template <bool KV>
__device__ __forceinline__ void sort_issue(SortSmem<KV> &S, int b, const uint64_t *kin,
                                           const uint32_t *vin, int64_t part, int64_t n) {
  const int64_t base = part * SORT_PART;
  const uint32_t cnt = (uint32_t)min((int64_t)SORT_PART, n - base);
  const uint32_t kb = (cnt & ~1u) * 8u;
  const uint32_t vb = KV ? (cnt & ~3u) * 4u : 0u;
  mbar_arrive_expect_tx(&S.bar[b], kb + vb);
  if (kb) bulk_g2s(S.keys[b], kin + base, kb, &S.bar[b]);
  if (KV && vb) bulk_g2s(S.vals[b], vin + base, vb, &S.bar[b]);
}

// One LSD pass over the 8-bit digit at bit `shift` of the stored words. Persistent CTAs take
// partitions of SORT_PART keys in claim order. KV: 64-bit keys with 32-bit values; otherwise
// packed words (key << idx_bits | value) only, and with `unpack` the pass writes the caller's
// keys (word >> idx_bits) and values (low idx_bits) instead of words.
template <bool KV>
__global__ void __launch_bounds__(SORT_THREADS, KV ? 2 : 3)
    onesweep_kernel(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                    uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                    const int64_t *n_int, int64_t capacity, int shift, int idx_bits, int unpack,
                    const uint32_t *hist, uint64_t *lb, uint64_t *lb_next,
                    uint32_t *part_counter, uint32_t *status, uint32_t wait_limit) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SortSmem<KV> &S = *reinterpret_cast<SortSmem<KV> *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // an earlier wait of the binning gave up: leave the keys alone (uniform over the launch, the
  // word was set before it started)
  if (binning_timed_out(status)) return;
  const int64_t n = min(*n_int, capacity);
  const int64_t nparts = (n + SORT_PART - 1) / SORT_PART;

  // clear the look-back entries the next pass will use (the previous pass is complete)
  for (int64_t e = (int64_t)blockIdx.x * SORT_THREADS + tid; e < nparts * 256;
       e += (int64_t)gridDim.x * SORT_THREADS)
    lb_next[e] = 0ull;

  uint32_t tot;
  {
    const uint32_t hx = block_excl_scan_256(hist[tid], S.warp_tmp, &tot);
    S.hist_excl[tid] = hx;
  }
  const uint32_t lt = lanemask_lt();
  const uint64_t vmask = (idx_bits >= 64) ? ~0ull : ((1ull << idx_bits) - 1ull);
  // Partitions are dealt round-robin (CTA c takes c, c + G, c + 2G, ...); the launch is
  // cooperative, so all CTAs are resident and a predecessor's CTA is always making progress.
  const int64_t G = gridDim.x;
  int64_t part = blockIdx.x;
  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
    if (part < nparts) sort_issue<KV>(S, 0, kin, vin, part, n);
  }
  __syncthreads();
  uint32_t phase = 0u;  // bit b = parity of buffer b's next phase
  int cur = 0;
  (void)part_counter;

  while (part < nparts) {
    const int64_t next = part + G;
    // prefetch this CTA's next partition into the other buffer
    if (tid == 0 && next < nparts) {
      fence_proxy_async_smem();
      sort_issue<KV>(S, cur ^ 1, kin, vin, next, n);
    }
    const bool ok = mbar_wait(&S.bar[cur], (phase >> cur) & 1u, status);
    phase ^= 1u << cur;
    if (__syncthreads_or(!ok)) {  // a copy never landed: drain (bounded) and leave
      if (next < nparts) mbar_wait(&S.bar[cur ^ 1], (phase >> (cur ^ 1)) & 1u, status);
      return;
    }
    const int64_t base = part * SORT_PART;
    const uint32_t cnt = (uint32_t)min((int64_t)SORT_PART, n - base);
    // ragged tail of the last partition: plain loads
    if (tid < 4) {
      const uint32_t kt = (cnt & ~1u) + tid;
      if (tid < 1 && kt < cnt) S.keys[cur][kt] = kin[base + kt];
      const uint32_t vt = (cnt & ~3u) + tid;
      if (KV && vt < cnt) S.vals[cur][vt] = vin[base + vt];
    }
    for (int e = tid; e < (SORT_THREADS / 32) * 256; e += SORT_THREADS) (&S.wcnt[0][0])[e] = 0u;
    __syncthreads();

    // load (warp-striped, order within a warp = k then lane = input order) and rank: warp
    // multi-split with match_any, stable
    uint64_t key[SORT_ITEMS];
    uint32_t val[SORT_ITEMS];
    uint32_t rank[SORT_ITEMS];
#pragma unroll
    for (int k = 0; k < SORT_ITEMS; ++k) {
      const uint32_t li = (uint32_t)(w * 32 * SORT_ITEMS + k * 32 + lane);
      const bool valid = li < cnt;
      key[k] = valid ? S.keys[cur][li] : 0ull;
      val[k] = (KV && valid) ? S.vals[cur][li] : 0u;
      const uint32_t d = valid ? (uint32_t)(key[k] >> shift) & 255u : 0x100u + lane;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t before = __popc(peers & lt);
      uint32_t c = 0;
      if (valid) c = S.wcnt[w][d];
      __syncwarp();
      if (valid && before == 0u) S.wcnt[w][d] = c + __popc(peers);
      __syncwarp();
      rank[k] = c + before;
    }
    __syncthreads();
    // per digit: per-warp exclusive offsets and the partition's count
    const int d = tid;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < SORT_THREADS / 32; ++ww) {
      const uint32_t c = S.wcnt[ww][d];
      S.wcnt[ww][d] = run;
      run += c;
    }
    const uint32_t dcount = run;
    uint64_t *my = lb + part * 256 + d;
    if (part == 0) st_volatile_u64(my, LB_INC | dcount);
    else st_volatile_u64(my, LB_AGG | dcount);
    uint32_t ptot;
    const uint32_t lstart = block_excl_scan_256(dcount, S.warp_tmp, &ptot);
    S.local_start[d] = lstart;
    uint64_t prefix = 0;
    if (part > 0) {
      prefix = look_back(lb + d, part, 256, status, wait_limit);
      st_volatile_u64(my, LB_INC | (prefix + dcount));
    }
    S.global_base[d] = S.hist_excl[d] + (uint32_t)prefix;
    __syncthreads();
    // local scatter into the partition's own buffer, sorted by digit
#pragma unroll
    for (int k = 0; k < SORT_ITEMS; ++k) {
      const uint32_t li = (uint32_t)(w * 32 * SORT_ITEMS + k * 32 + lane);
      if (li < cnt) {
        const uint32_t dd = (uint32_t)(key[k] >> shift) & 255u;
        const uint32_t pos = S.local_start[dd] + S.wcnt[w][dd] + rank[k];
        S.keys[cur][pos] = key[k];
        if (KV) S.vals[cur][pos] = val[k];
      }
    }
    __syncthreads();
    // global scatter: consecutive shared positions of one digit go to consecutive addresses
    for (uint32_t i = tid; i < cnt; i += SORT_THREADS) {
      const uint64_t kk = S.keys[cur][i];
      const uint32_t dd = (uint32_t)(kk >> shift) & 255u;
      const uint64_t gpos = (uint64_t)S.global_base[dd] + (i - S.local_start[dd]);
      if (gpos < (uint64_t)n) {
        if (KV) {
          kout[gpos] = kk;
          vout[gpos] = S.vals[cur][i];
        } else if (unpack) {
          kout[gpos] = kk >> idx_bits;
          vout[gpos] = (uint32_t)(kk & vmask);
        } else {
          kout[gpos] = kk;
        }
      }
    }
    __syncthreads();  // buffer, counters and offsets are reused by the next partition
    part = next;
    cur ^= 1;
  }
}

// Tile ids come from the sorted keys; they are checked against the tile count so that keys
// left undefined by a device-side error cannot steer a write out of bounds.
__global__ void ranges_kernel(const uint64_t *__restrict__ keys, const int64_t *n_int,
                              int64_t capacity, int64_t total_tiles,
                              uint32_t *__restrict__ ranges, uint32_t *status) {
  if (binning_timed_out(status)) return;
  const int64_t n = min(*n_int, capacity);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t t = keys[i] >> 32;
    // the dropped pairs carry tile id total_tiles; any larger id is an error (checked build)
    if (t >= (uint64_t)total_tiles) {
      in_bounds(t, (uint64_t)total_tiles + 1u, status);
      continue;
    }
    if (i == 0 || (keys[i - 1] >> 32) != t) ranges[2 * t] = (uint32_t)i;
    if (i == n - 1 || (keys[i + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(i + 1);
  }
}

// The pairs dropped at emission (beyond their record's rect) sorted to the end: the result
// counts the kept pairs only, unless the candidates overflowed the capacity (the count then
// stays the candidates', for the caller to grow the buffers).
__global__ void drop_count_kernel(int64_t *n_int, int64_t capacity,
                                  const unsigned long long *n_dropped, const uint32_t *status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && !binning_timed_out(status) && *n_int <= capacity)
    *n_int -= (int64_t)*n_dropped;
}

}  // namespace

cudaError_t launch_bin_sort_onesweep(const fgs_record *records, const uint32_t *tiles_touched,
                                     int64_t n, const Views &vs, uint64_t *keys,
                                     uint32_t *vals, int64_t capacity, uint32_t *tile_ranges,
                                     int64_t *n_int, char *ws, const WsLayout &L,
                                     const CallOpts &opt, cudaStream_t st) {
  cudaError_t e;
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.header);
  uint64_t *scan_lb = reinterpret_cast<uint64_t *>(ws + L.scan_lb);
  uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.sort_hist);
  uint64_t *sort_lb = reinterpret_cast<uint64_t *>(ws + L.sort_lb);
  uint64_t *alt_keys = reinterpret_cast<uint64_t *>(ws + L.words);
  uint32_t *alt_vals = reinterpret_cast<uint32_t *>(ws + L.alt_vals);
  const int64_t R = (int64_t)vs.n * n;
  // tile ids 0 .. total_tiles (the last one marks the pairs dropped at emission)
  int sort_tile_bits = 0;
  while (sort_tile_bits < 32 && ((int64_t)1 << sort_tile_bits) <= vs.total_tiles) ++sort_tile_bits;
  const int passes = (32 + sort_tile_bits + 7) / 8;
  unsigned long long *n_dropped = &hdr->n_dropped;

  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * SORT_MAX_PASSES * 256, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)vs.total_tiles, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(sort_lb, 0, sizeof(uint64_t) * 256 * (size_t)L.sort_parts, st)) != cudaSuccess) return e;
  if (R == 0) return cudaMemsetAsync(n_int, 0, sizeof(int64_t), st);
  if ((e = cudaMemsetAsync(scan_lb, 0, sizeof(uint64_t) * 2 * (size_t)L.scan_parts, st)) != cudaSuccess) return e;

  // Packed mode when (tile << 32 | depth) << idx_bits | record fits in 64 bits: the passes
  // move 8-byte words instead of 12-byte pairs and the last pass unpacks into the caller's
  // keys and values. The ping-pong is arranged so that the last pass never reads the buffer
  // it writes.
  int idx_bits = 0;
  while (idx_bits < 32 && ((int64_t)1 << idx_bits) < R) ++idx_bits;
  const bool packed = idx_bits + 32 + sort_tile_bits <= 64;
  uint64_t *k0, *k1;
  uint32_t *v0 = nullptr, *v1 = nullptr;
  if (packed) {
    const bool last_even = ((passes - 1) & 1) == 0;  // last pass reads k0 if even
    k0 = last_even ? alt_keys : keys;
    k1 = last_even ? keys : alt_keys;
  } else {
    k0 = (passes & 1) ? alt_keys : keys;
    v0 = (passes & 1) ? alt_vals : vals;
    k1 = (passes & 1) ? keys : alt_keys;
    v1 = (passes & 1) ? vals : alt_vals;
  }

  uint32_t *vis_rec = reinterpret_cast<uint32_t *>(ws + L.vis_rec);
  uint64_t *vis_off = reinterpret_cast<uint64_t *>(ws + L.vis_off);
  uint32_t *chunk_first = reinterpret_cast<uint32_t *>(ws + L.chunk_first);
  scan_kernel<<<(unsigned)L.scan_parts, EMIT_THREADS, 0, st>>>(
      tiles_touched, R, capacity, n_int, &hdr->n_candidates, &hdr->n_visible, scan_lb,
      scan_lb + L.scan_parts, &hdr->scan_parts, vis_rec, vis_off, chunk_first, &hdr->status,
      opt.wait_limit);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int64_t egrid = (int64_t)sm_count() * 4;
  if (egrid > L.chunks) egrid = L.chunks;
  if (egrid < 1) egrid = 1;
  emit_kernel<<<(unsigned)egrid, EMIT_THREADS, 0, st>>>(
      records, n, vs, vis_rec, vis_off, chunk_first, n_int, &hdr->n_visible, k0, v0, capacity,
      hist, passes, idx_bits, packed ? 1 : 0, n_dropped, &hdr->status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  static int occ_kv = 0, occ_packed = 0;
  const size_t smem_kv = sizeof(SortSmem<true>), smem_packed = sizeof(SortSmem<false>);
  if (occ_kv == 0) {
    if ((e = cudaFuncSetAttribute(onesweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_kv)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(onesweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_packed)) != cudaSuccess)
      return e;
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, onesweep_kernel<true>, SORT_THREADS, smem_kv);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, onesweep_kernel<false>, SORT_THREADS, smem_packed);
    occ_kv = a > 0 ? a : 1;
    occ_packed = b > 0 ? b : 1;
  }
  int64_t grid = (int64_t)sm_count() * (packed ? occ_packed : occ_kv);
  if (grid > L.sort_parts) grid = L.sort_parts;
  if (grid < 1) grid = 1;
  for (int p = 0; p < passes; ++p) {
    const uint64_t *kin = (p & 1) ? k1 : k0;
    uint64_t *kout = (p & 1) ? k0 : k1;
    uint64_t *lb = sort_lb + (size_t)(p & 1) * 256 * (size_t)L.sort_parts;
    uint64_t *lbn = sort_lb + (size_t)((p + 1) & 1) * 256 * (size_t)L.sort_parts;
    if (packed) {
      const bool last = p == passes - 1;
      const uint64_t *a0 = kin;
      const uint32_t *a1 = nullptr;
      uint64_t *a2 = last ? keys : kout;
      uint32_t *a3 = last ? vals : nullptr;
      int a6 = idx_bits + 8 * p, a7 = idx_bits, a8 = last ? 1 : 0;
      const uint32_t *a9 = hist + p * 256;
      uint32_t *a12 = &hdr->tile_parts, *a13 = &hdr->status;
      uint32_t a14 = opt.wait_limit;
      void *args[] = {&a0, &a1, &a2, &a3, &n_int, &capacity, &a6, &a7, &a8, &a9, &lb, &lbn,
                      &a12, &a13, &a14};
      e = cudaLaunchCooperativeKernel((const void *)onesweep_kernel<false>, dim3((unsigned)grid),
                                      dim3(SORT_THREADS), args, smem_packed, st);
      if (e != cudaSuccess) return e;
    } else {
      const uint32_t *vin = (p & 1) ? v1 : v0;
      uint32_t *vout = (p & 1) ? v0 : v1;
      int a6 = 8 * p, a7 = 0, a8 = 0;
      const uint32_t *a9 = hist + p * 256;
      uint32_t *a12 = &hdr->tile_parts, *a13 = &hdr->status;
      uint32_t a14 = opt.wait_limit;
      void *args[] = {&kin, &vin, &kout, &vout, &n_int, &capacity, &a6, &a7, &a8, &a9, &lb, &lbn,
                      &a12, &a13, &a14};
      e = cudaLaunchCooperativeKernel((const void *)onesweep_kernel<true>, dim3((unsigned)grid),
                                      dim3(SORT_THREADS), args, smem_kv, st);
      if (e != cudaSuccess) return e;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int64_t rgrid = (int64_t)sm_count() * 8;
  ranges_kernel<<<(unsigned)rgrid, 256, 0, st>>>(keys, n_int, capacity, vs.total_tiles,
                                                  tile_ranges, &hdr->status);
  drop_count_kernel<<<1, 32, 0, st>>>(n_int, capacity, n_dropped, &hdr->status);
  return cudaGetLastError();
}

}  // namespace fgs
