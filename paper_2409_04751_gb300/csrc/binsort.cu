// binsort.cu - tile binning and key sort (Sec. 3.1 "Rendering"; Sec. 4.1 duplicateWithKeys and
// radixSort), sm_103a.
//
// The result is the one the method defines: for every (record, tile) pair of a record's tile
// rect, key = tile << 32 | depth bits and value = record, stably sorted by key, and each tile's
// [start, end) in the sorted arrays. Instead of emitting every pair and sorting them all (the
// device-wide radix sort over all key bits is kept in onesweep.cu as the option
// FGS_BIN_ONESWEEP), the records are binned into cells of CELL x CELL tiles, each cell's short
// list is sorted once by (depth, record), and every tile takes its pairs out of its cell's
// sorted list in order:
//
//  1. cell_count_kernel: the number of rect pairs and of visible records, and per cell the
//     records with a pair in it. A warp numbers the cells of its 32 records and takes them 32
//     at a time (the same work per lane however large the records); they are counted in shared
//     memory, with one global atomic per CTA and cell.
//  2. tile_scan_kernel over the cells: exclusive scan of the cell counts (decoupled look-back)
//     gives every cell's start; cells are listed by size class.
//  3. cell_scatter_kernel: the same walk writes depth bits << 32 | record into the record's
//     cells (slots claimed per CTA and cell, then per entry in shared memory), each with the
//     mask of the cell's tiles that hold one of its pairs (exact binning: whose pixels its
//     alpha >= 1/255 ellipse reaches).
//  4. cell_sort_kernel (one launch per size class): each cell's list is sorted in shared memory
//     with its masks (a one-pass bucket sort on the depth bits, or LSD radix passes when the
//     depths are too clustered for it), in place, and the cell's tiles get their pair counts.
//  5. tile_scan_kernel over the tiles: exclusive scan of the tile counts gives every tile's
//     [start, end) and the number of pairs.
//  6. cell_emit_kernel: one CTA per cell stages the cell's sorted list in shared memory and
//     one warp per tile keeps, in order, the entries whose mask has the tile's bit: the tile's
//     pairs, already sorted; they are written out as keys and values.
// A record's cells are about a seventh of its tiles on the 180-degree workloads, so the sort
// handles a seventh of the pairs, no per-pair atomic is issued, and the pairs are written once.
// The number of valid pairs is read on the device, so nothing here needs a host sync.
#include "fgs_internal.cuh"
#include "scan.cuh"

namespace fgs {

namespace {

constexpr int REC_THREADS = 256;
constexpr int REC_PER_THREAD = 4;
constexpr int REC_BLOCK = REC_THREADS * REC_PER_THREAD;  // records per CTA of the cell walks
constexpr int SMEM_CELLS = CELL_WALK_SMEM;  // cell counters a CTA keeps in shared memory (else global)
static_assert(REC_BLOCK == CELL_WALK_BLOCK, "the workspace sizes the count table by this block");
constexpr int CELL_CAP0 = 4096;   // cells of at most this many entries: the smaller sort class

// The pairs of one record: the first k = min(tiles_touched, w h) tiles of its w x h rect in
// row-major order, i.e. fr full rows from row y0 and the first rem tiles of the next row.
struct PairSet {
  uint32_t x0, y0, x1;
  uint32_t fr, rem;
  uint32_t k;
};

// false for a record with no pairs (tiles_touched = 0, or a rect outside its view's grid)
__device__ __forceinline__ bool pair_set(uint4 w2, uint32_t tt, const View &V, PairSet &P) {
  const uint32_t x0 = w2.z & 0xffffu, y0 = w2.z >> 16, x1 = w2.w & 0xffffu, y1 = w2.w >> 16;
  if (tt == 0u || !(x0 <= x1 && y0 <= y1 && x1 < (uint32_t)V.tiles_x && y1 < (uint32_t)V.tiles_y))
    return false;
  const uint32_t w = x1 - x0 + 1u, h = y1 - y0 + 1u;
  P.k = (uint32_t)min((uint64_t)tt, (uint64_t)w * h);
  P.x0 = x0; P.y0 = y0; P.x1 = x1;
  P.fr = P.k / w;
  P.rem = P.k - P.fr * w;
  return true;
}

// The cells holding at least one of a record's pairs, numbered: first the cells of the full
// rows (cols x rows, row-major from (cx0, cy0)), then the cells of the partial row (row cyB,
// colsB cells from cx0) that the full rows' cells do not already cover. Each holds a pair, so
// a record has at most as many cells as pairs.
struct CellSet {
  uint32_t cx0, cy0, cols, rows;
  uint32_t cyB, colsB;
  uint32_t n;
};

__device__ __forceinline__ CellSet cell_set(const PairSet &P) {
  CellSet S;
  S.cx0 = P.x0 / CELL;
  S.cy0 = P.y0 / CELL;
  S.cols = P.x1 / CELL - S.cx0 + 1u;
  uint32_t last = 0xffffffffu;
  S.rows = 0u;
  if (P.fr > 0u) {
    last = (P.y0 + P.fr - 1u) / CELL;
    S.rows = last - S.cy0 + 1u;
  }
  S.cyB = (P.y0 + P.fr) / CELL;
  S.colsB = P.rem > 0u && S.cyB != last ? (P.x0 + P.rem - 1u) / CELL - S.cx0 + 1u : 0u;
  S.n = S.cols * S.rows + S.colsB;
  return S;
}

// Walks the cells of 32 consecutive records [r0, r0 + 32) with one warp: lane l loads record
// r0 + l (calling g(pairs) if it has any), the warp numbers all their cells in record order
// and takes them 32 at a time, lane l calling f(record, view, depth bits, cx, cy, pairs) for
// cell e0 + l (pairs without k). Every lane does the same work
// however the cells are spread over the records.
template <class G, class F>
__device__ __forceinline__ void warp_cells(const fgs_record *__restrict__ rec,
                                           const uint32_t *__restrict__ tt, int64_t r0, int64_t R,
                                           int64_t n_per_view, const Views &vs, G g, F f) {
  const int lane = threadIdx.x & 31;
  const int64_t r = r0 + lane;
  CellSet S{};
  PairSet P{};
  int view = 0;
  uint32_t depth = 0u;
  if (r < R) {
    const uint32_t t = tt[r];
    if (t != 0u) {
      view = (int)((uint32_t)r / (uint32_t)n_per_view);  // R < 2^32
      const uint4 w2 = __ldg(reinterpret_cast<const uint4 *>(rec + r) + 2);
      if (pair_set(w2, t, vs.v[view], P)) {
        S = cell_set(P);
        depth = w2.y;
        g(P);
      }
    }
  }
  uint32_t incl = S.n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  const uint32_t first = incl - S.n;
  for (uint32_t e0 = 0; e0 < total; e0 += 32u) {
    const uint32_t e = e0 + (uint32_t)lane;
    // owner: the number of lanes whose cells all come before e
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint32_t v = __shfl_sync(0xffffffffu, incl, j + step - 1);
      if (v <= e) j += step;
    }
    const uint32_t i = e - __shfl_sync(0xffffffffu, first, j);
    const uint32_t cx0 = __shfl_sync(0xffffffffu, S.cx0, j);
    const uint32_t cy0 = __shfl_sync(0xffffffffu, S.cy0, j);
    const uint32_t cols = __shfl_sync(0xffffffffu, S.cols, j);
    const uint32_t rows = __shfl_sync(0xffffffffu, S.rows, j);
    const uint32_t cyB = __shfl_sync(0xffffffffu, S.cyB, j);
    const int vj = __shfl_sync(0xffffffffu, view, j);
    const uint32_t dj = __shfl_sync(0xffffffffu, depth, j);
    PairSet Pj;
    const uint32_t xy = __shfl_sync(0xffffffffu, P.x0 | (P.y0 << 16), j);
    const uint32_t fr_rem = __shfl_sync(0xffffffffu, P.fr | (P.rem << 16), j);
    Pj.x0 = xy & 0xffffu;
    Pj.y0 = xy >> 16;
    Pj.x1 = __shfl_sync(0xffffffffu, P.x1, j);
    Pj.fr = fr_rem & 0xffffu;
    Pj.rem = fr_rem >> 16;
    Pj.k = 0u;
    if (e < total) {
      const uint32_t nb = cols * rows;
      uint32_t cx, cy;
      if (i < nb) {
        const uint32_t q = i / cols;
        cy = cy0 + q;
        cx = cx0 + (i - q * cols);
      } else {
        cy = cyB;
        cx = cx0 + (i - nb);
      }
      f(r0 + j, vj, dj, cx, cy, Pj);
    }
  }
}

// Bits lo - b .. hi - b of [lo, hi] clipped to the cell span [b, b + CELL) (0 if disjoint).
__device__ __forceinline__ uint32_t span_bits(uint32_t lo, uint32_t hi, uint32_t b) {
  const uint32_t l = max(lo, b), h = min(hi, b + (CELL - 1));
  return l <= h ? (2u << (h - b)) - (1u << (l - b)) : 0u;
}

// The record's pairs inside the cell whose first tile is (bx, by): bit ly * CELL + lx for
// the tile (bx + lx, by + ly).
__device__ __forceinline__ uint32_t cell_mask(const PairSet &P, uint32_t bx, uint32_t by) {
  uint32_t m = 0u;
  if (P.fr > 0u) {
    const uint32_t cols = span_bits(P.x0, P.x1, bx);
    const uint32_t rows = span_bits(P.y0, P.y0 + P.fr - 1u, by);
#pragma unroll
    for (int ly = 0; ly < CELL; ++ly)
      if ((rows >> ly) & 1u) m |= cols << (CELL * ly);
  }
  if (P.rem > 0u) {
    const uint32_t y = P.y0 + P.fr;
    if (y >= by && y < by + CELL) m |= span_bits(P.x0, P.x0 + P.rem - 1u, bx) << (CELL * (y - by));
  }
  return m;
}

// Exact binning: the tiles of mask m (cell at tile (bx, by)) that the record's alpha >= 1/255
// ellipse reaches.
__device__ __forceinline__ uint32_t ellipse_mask(const fgs_record *rp, uint32_t m, uint32_t bx,
                                                 uint32_t by) {
  if (m == 0u) return 0u;
  const float4 w0 = __ldg(reinterpret_cast<const float4 *>(rp));
  const float4 w1 = __ldg(reinterpret_cast<const float4 *>(rp) + 1);
  const EllipseTest E = ellipse_test(w0.x, w0.y, w0.z, w0.w, w1.x,
                                     fmaxf(2.f * logf(255.f * w1.y), 0.f));
  for (uint32_t rest = m; rest; rest &= rest - 1u) {
    const uint32_t b = __ffs(rest) - 1;
    const float xl = (float)((bx + b % CELL) * TILE) + 0.5f;
    const float yl = (float)((by + b / CELL) * TILE) + 0.5f;
    if (!ellipse_reaches_tile(E, xl, xl + (TILE - 1), yl, yl + (TILE - 1))) m &= ~(1u << b);
  }
  return m;
}

__device__ __forceinline__ int64_t cell_id(const View &V, uint32_t cx, uint32_t cy) {
  return V.cell_offset + (int64_t)cy * V.cells_x + cx;
}

// Step 1. Per-cell entry counts (cell_ranges[2c]), rect pairs (*n_cand) and visible records;
// with cta_counts, also each CTA's own counts per cell (row blockIdx of the table).
__global__ void __launch_bounds__(REC_THREADS)
    cell_count_kernel(const fgs_record *__restrict__ rec, const uint32_t *__restrict__ tt,
                      int64_t R, int64_t n_per_view, Views vs, int64_t capacity,
                      uint32_t *cell_ranges, uint32_t *__restrict__ cta_counts,
                      unsigned long long *n_cand, unsigned long long *n_vis, uint32_t *status) {
  __shared__ uint32_t s_cnt[SMEM_CELLS];
  __shared__ unsigned long long s_sum[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool in_smem = vs.total_cells <= SMEM_CELLS;
  if (FGS_CHECK && blockIdx.x == 0 && tid == 0) {  // the rasterizers' index bounds
    WsHeader *h = reinterpret_cast<WsHeader *>(status);
    h->bounds_records = (uint32_t)R;
    h->bounds_pairs = (uint32_t)capacity;
    h->bounds_magic = BOUNDS_MAGIC;
  }
  if (in_smem)
    for (int c = tid; c < (int)vs.total_cells; c += REC_THREADS) s_cnt[c] = 0u;
  if (tid < 2) s_sum[tid] = 0ull;
  __syncthreads();
  unsigned long long pairs = 0, vis = 0;
  const int64_t base = (int64_t)blockIdx.x * REC_BLOCK;
  for (int i = 0; i < REC_PER_THREAD; ++i) {
    const int64_t r0 = base + (int64_t)(i * (REC_THREADS / 32) + wid) * 32;
    if (r0 >= R) break;
    warp_cells(rec, tt, r0, R, n_per_view, vs,
               [&](const PairSet &P) {
                 pairs += P.k;
                 ++vis;
               },
               [&](int64_t, int v, uint32_t, uint32_t cx, uint32_t cy, const PairSet &) {
                 const int64_t c = cell_id(vs.v[v], cx, cy);
                 if (in_smem) atomicAdd(&s_cnt[c], 1u);
                 else atomicAdd(&cell_ranges[2 * c], 1u);
               });
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    vis += __shfl_xor_sync(0xffffffffu, vis, o);
  }
  if (lane == 0) {
    atomicAdd(&s_sum[0], pairs);
    atomicAdd(&s_sum[1], vis);
  }
  __syncthreads();
  if (in_smem) {
    uint32_t *row = cta_counts ? cta_counts + (size_t)blockIdx.x * vs.total_cells : nullptr;
    for (int c = tid; c < (int)vs.total_cells; c += REC_THREADS) {
      const uint32_t v = s_cnt[c];
      if (v) atomicAdd(&cell_ranges[2 * c], v);
      if (row) row[c] = v;  // this CTA's counts, for the scatter
    }
  }
  if (tid == 0) {
    if (s_sum[0]) atomicAdd(n_cand, s_sum[0]);
    if (s_sum[1]) atomicAdd(n_vis, s_sum[1]);
  }
}

// Step 3. Writes depth bits << 32 | record into every cell of every record (cell_ranges[2c + 1]
// holds the cell's next free slot, set to its start by the cell scan), and beside it the mask
// of the cell's tiles that hold one of the record's pairs (exact binning: those its alpha >=
// 1/255 ellipse reaches; a mask can then be empty). With the cell counters
// in shared memory a CTA takes its entries per cell from the count table of the cell walk (or,
// without the table, counts them again), claims a block of slots per cell with one global
// atomic, and hands the slots out in shared memory; the order inside a cell is irrelevant (the
// cell is sorted next).
template <bool ELLIPSE>
__global__ void __launch_bounds__(REC_THREADS)
    cell_scatter_kernel(const fgs_record *__restrict__ rec, const uint32_t *__restrict__ tt,
                        int64_t R, int64_t n_per_view, Views vs, uint32_t *cell_ranges,
                        uint64_t *__restrict__ words, uint16_t *__restrict__ masks,
                        const uint32_t *__restrict__ cta_counts,
                        const unsigned long long *n_cand, int64_t capacity, uint32_t *status) {
  __shared__ uint32_t s_cnt[SMEM_CELLS];
  if (binning_timed_out(status) || (int64_t)*n_cand > capacity) return;
  const int tid = threadIdx.x, wid = tid >> 5;
  const bool in_smem = vs.total_cells <= SMEM_CELLS;
  const int64_t base = (int64_t)blockIdx.x * REC_BLOCK;
  if (in_smem && cta_counts) {
    // the counts of this CTA's records, as the cell walk found them (same CTA-to-record map)
    const uint32_t *row = cta_counts + (size_t)blockIdx.x * vs.total_cells;
    for (int c = tid; c < (int)vs.total_cells; c += REC_THREADS) s_cnt[c] = row[c];
    __syncthreads();
  } else if (in_smem) {
    for (int c = tid; c < (int)vs.total_cells; c += REC_THREADS) s_cnt[c] = 0u;
    __syncthreads();
    for (int i = 0; i < REC_PER_THREAD; ++i) {
      const int64_t r0 = base + (int64_t)(i * (REC_THREADS / 32) + wid) * 32;
      if (r0 >= R) break;
      warp_cells(rec, tt, r0, R, n_per_view, vs, [](const PairSet &) {},
                 [&](int64_t, int v, uint32_t, uint32_t cx, uint32_t cy, const PairSet &) {
                   atomicAdd(&s_cnt[cell_id(vs.v[v], cx, cy)], 1u);
                 });
    }
    __syncthreads();
  }
  if (in_smem) {
    // the block's slots of each cell; s_cnt then holds the next one to hand out
    for (int c = tid; c < (int)vs.total_cells; c += REC_THREADS)
      if (s_cnt[c]) s_cnt[c] = atomicAdd(&cell_ranges[2 * c + 1], s_cnt[c]);
    __syncthreads();
  }
  for (int i = 0; i < REC_PER_THREAD; ++i) {
    const int64_t r0 = base + (int64_t)(i * (REC_THREADS / 32) + wid) * 32;
    if (r0 >= R) break;
    warp_cells(rec, tt, r0, R, n_per_view, vs, [](const PairSet &) {},
               [&](int64_t r, int v, uint32_t depth, uint32_t cx, uint32_t cy, const PairSet &P) {
      const int64_t c = cell_id(vs.v[v], cx, cy);
      const uint32_t slot = in_smem ? atomicAdd(&s_cnt[c], 1u) : atomicAdd(&cell_ranges[2 * c + 1], 1u);
      const uint32_t bx = cx * CELL, by = cy * CELL;
      uint32_t m = cell_mask(P, bx, by);
      if (ELLIPSE) m = ellipse_mask(rec + r, m, bx, by);
      // a record's cells never outnumber its pairs, so the entries fit the capacity (checked
      // build: verified)
      if (in_bounds(slot, (uint64_t)capacity, status) && (int64_t)slot < capacity) {
        words[slot] = ((uint64_t)depth << 32) | (uint64_t)r;
        masks[slot] = (uint16_t)m;
      }
    });
  }
}

// Steps 2 and 5. Exclusive scan of per-segment counts (ranges[2s], s a cell or a tile) in
// segment order, with decoupled look-back over partitions of TSCAN_PART segments.
// Cells (FINAL = false): writes ranges[s] = (start, start) for every non-empty cell (the second
// word is the scatter's cursor and ends as the cell's end) and appends the cell to the list of
// its size class (at most cls_cap entries: class 0); empty cells keep (0, 0). Tiles (FINAL =
// true): writes ranges[s] = (start, end) for every tile, (0, 0) when empty, and the
// number of pairs to *n_int (the rect count instead when it exceeds the capacity, so the caller
// can grow the buffers). A tile's count was written by the sort of its cell, so the tiles of an
// empty cell (cell_ranges (0, 0): no sort ran for it) count zero whatever their count word
// holds, and the tile ranges need no clearing beforehand. It runs even after a look-back of
// the binning gave up (its counts are then all zero), so that every partition publishes and no
// wait of its own look-back depends on a partition that left early.
template <bool FINAL>
__global__ void __launch_bounds__(256)
    tile_scan_kernel(uint32_t *ranges, int64_t total, uint64_t *lb, uint32_t *part_counter,
                     uint32_t *lists, uint32_t *seg_count, uint32_t cls_cap,
                     const unsigned long long *n_cand, int64_t capacity, int64_t *n_int,
                     uint32_t *status, uint32_t wait_limit, Views vs,
                     const uint32_t *__restrict__ cell_ranges) {
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
  // with more rect pairs than capacity nothing was binned: read the counts as zero, and report
  // the overflow (the caller grows the buffers from the pair count)
  const bool fits = (int64_t)*n_cand <= capacity;
  if (!fits && part == 0 && tid == 0) set_status(status, ST_CAPACITY);
  // after a look-back of the binning gave up no sort wrote the tile counts: read them as zero
  const bool counts_ok = fits && !(FINAL && binning_timed_out(status));
  constexpr int ITEMS = TSCAN_PART / 256;
  uint32_t c[ITEMS];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int64_t s = base + tid * ITEMS + k;
    bool live = s < total && counts_ok;
    if (FINAL && live) {  // the tile's cell was sorted (non-empty) or its count is zero
      const View &V = vs.v[view_of_tile(vs, s)];
      const int64_t local = s - V.tile_offset;
      const int64_t ty = local / V.tiles_x, tx = local - ty * V.tiles_x;
      const int64_t cell = V.cell_offset + (ty / CELL) * V.cells_x + tx / CELL;
      const uint2 crg = __ldg(reinterpret_cast<const uint2 *>(cell_ranges) + cell);
      live = crg.y > crg.x;
    }
    c[k] = live ? ranges[2 * s] : 0u;
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
    if (FINAL && base + TSCAN_PART >= total)
      *n_int = (int64_t)*n_cand <= capacity ? (int64_t)(prefix + agg) : (int64_t)*n_cand;
  }
  uint32_t cls_rank[ITEMS];
  if (!FINAL) {  // class ranks inside the CTA (order within a class list is irrelevant)
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int cls = c[k] <= cls_cap ? 0 : 1;
      cls_rank[k] = c[k] > 0u ? atomicAdd(&s_cls[cls], 1u) : 0u;
    }
  }
  __syncthreads();
  if (!FINAL && tid < 2) s_cls_base[tid] = s_cls[tid] ? atomicAdd(&seg_count[tid], s_cls[tid]) : 0u;
  __syncthreads();
  uint64_t o = s_prefix + off;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int64_t s = base + tid * ITEMS + k;
    if (FINAL && s < total && c[k] == 0u) {  // an empty tile: (0, 0)
      ranges[2 * s] = 0u;
      ranges[2 * s + 1] = 0u;
    }
    if (c[k] > 0u) {
      ranges[2 * s] = (uint32_t)o;
      ranges[2 * s + 1] = (uint32_t)(FINAL ? o + c[k] : o);
      if (!FINAL) {
        const int cls = c[k] <= cls_cap ? 0 : 1;
        lists[(size_t)cls * (size_t)total + s_cls_base[cls] + cls_rank[k]] = (uint32_t)s;
      }
    }
    o += c[k];
  }
}

// Segment sort. A cell's list holds its words depth_bits << 32 | record in arbitrary order;
// sorting the words as 64-bit integers orders them by depth and breaks depth ties by record
// index, which is the order a stable sort of the keys (tile << 32 | depth) in emission order
// gives inside every tile. LSD radix passes over 8-bit digits, skipping digits that are equal in
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
  uint16_t pay[CAP];  // each word's 16-bit payload (its tile mask), moved with it
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
__device__ __forceinline__ void smem_pass(SegSmem<NT, CAP> &S, uint64_t (&x)[IPT],
                                          uint32_t (&p)[IPT], uint32_t cnt, int shift) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t rank[IPT];
  rank_items<NT, IPT, CAP>(S, x, cnt, shift, rank);
  digit_offsets<NT, IPT, CAP>(S);
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    if (li < cnt) {
      const uint32_t d = (uint32_t)(x[k] >> shift) & 255u;
      const uint32_t pos = S.dstart[d] + S.rx.wcnt[w][d] + rank[k];
      S.buf[pos] = x[k];
      S.pay[pos] = (uint16_t)p[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    x[k] = li < cnt ? S.buf[li] : 0ull;
    p[k] = li < cnt ? (uint32_t)S.pay[li] : 0u;
  }
}

// Sort one segment of cnt <= NT * IPT words with their payloads in shared memory and write
// them to out / pout (which may be src / psrc: everything is read before the first write).
template <int NT, int IPT, int CAP>
__device__ __forceinline__ void sort_segment_smem(SegSmem<NT, CAP> &S, const uint64_t *src,
                                                  const uint16_t *psrc, uint32_t cnt,
                                                  uint64_t *out, uint16_t *pout) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // the lane masks share storage with the bucket sort's counters: clear them first
  for (int e = threadIdx.x; e < (NT / 32) * 256; e += NT) (&S.rx.wmask[0][0])[e] = 0u;
  __syncthreads();
  uint64_t x[IPT];
  uint32_t p[IPT];
  uint64_t a = ~0ull, o = 0ull;
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    x[k] = li < cnt ? src[li] : 0ull;
    p[k] = li < cnt ? (uint32_t)psrc[li] : 0u;
    if (li < cnt) {
      S.buf[li] = x[k];
      a &= x[k];
      o |= x[k];
    }
  }
  block_and_or<NT, IPT, CAP>(S, a, o);
  const uint64_t varying = a ^ o;
#pragma unroll
  for (int d = 4; d < 8; ++d)
    if ((varying >> (8 * d)) & 255u) smem_pass<NT, IPT, CAP>(S, x, p, cnt, 8 * d);
  // equal depths (the high halves) in adjacent slots: sort again over every digit
  bool tie = false;
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    if (li + 1 < cnt) tie |= (S.buf[li] >> 32) == (S.buf[li + 1] >> 32);
  }
  if (__syncthreads_or(tie)) {
#pragma unroll
    for (int d = 0; d < 8; ++d)
      if ((varying >> (8 * d)) & 255u) smem_pass<NT, IPT, CAP>(S, x, p, cnt, 8 * d);
  }
  // without a radix pass (one word) the payload is still in registers only
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(w * 32 * IPT + k * 32 + lane);
    if (li < cnt) S.pay[li] = (uint16_t)p[k];
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += NT) {
    out[i] = S.buf[i];
    pout[i] = S.pay[i];
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
                                                    const uint16_t *psrc, uint32_t cnt,
                                                    uint64_t *out, uint16_t *pout) {
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
    if (li < cnt) S.pay[li] = psrc[li];  // staged by original slot, placed at the end
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
  uint32_t p[IPT];
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(k * NT + tid);
    p[k] = li < cnt ? (uint32_t)S.pay[li] : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const uint32_t li = (uint32_t)(k * NT + tid);
    if (li < cnt) {
      S.buf[bs[k]] = x[k];
      S.pay[bs[k]] = (uint16_t)p[k];
    }
  }
  __syncthreads();
  for (uint32_t i = tid; i < cnt; i += NT) {
    out[i] = S.buf[i];
    pout[i] = S.pay[i];
  }
  __syncthreads();  // buf and counters reused by the next segment
  return true;
}

// Sort one segment longer than NT * IPT through global memory: per digit, a histogram pass
// over the segment, then the segment in chunks of NT * IPT words in order, each ranked in
// shared memory and scattered to its place in the other buffer (words <-> scratch). All digits
// with varying bits are sorted. The last step copies the words back to `words` if they ended in
// the scratch buffer.
template <int NT, int IPT, int CAP>
__device__ __noinline__ void sort_segment_chunked(SegSmem<NT, CAP> &S, uint64_t *words,
                                                  uint32_t cnt, uint64_t *scratch) {
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
  uint64_t *src = words, *dst = scratch;
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
  if (src != words)
    for (uint32_t i = tid; i < cnt; i += NT) words[i] = src[i];
  __syncthreads();
}

// The radix path kept out of line for the large classes, where inlining it would raise the
// register needs of the bucket sort that every segment takes first.
template <int NT, int IPT, int CAP>
__device__ __noinline__ void sort_segment_smem_outlined(SegSmem<NT, CAP> &S, uint64_t *words,
                                                        uint16_t *pay, uint32_t cnt) {
  sort_segment_smem<NT, IPT, CAP>(S, words, pay, cnt, words, pay);
}

// Sort one segment of cnt <= NT * IPT words in shared memory: the bucket sort, or the radix
// passes if the bucket sort declines.
template <int NT, int IPT, int CAP>
__device__ __forceinline__ void sort_segment(SegSmem<NT, CAP> &S, uint64_t *words, uint16_t *pay,
                                             uint32_t cnt) {
  if (bucket_sort_segment<NT, IPT, CAP>(S, words, pay, cnt, words, pay)) return;
  if constexpr (CAP <= SEG_CAP0)
    sort_segment_smem<NT, IPT, CAP>(S, words, pay, cnt, words, pay);
  else
    sort_segment_smem_outlined<NT, IPT, CAP>(S, words, pay, cnt);
}

// Step 4. One CTA per listed cell of a size class, persistent over the class list: sorts the
// cell's words in place, each with its tile mask (the number of words per thread picked per
// cell, the smallest of IPT_LO and 2 IPT_LO that holds it; cells longer than CAP are sorted in
// chunks through the scratch buffer, and their masks found again from the records afterwards),
// then writes the pair count of each of the cell's tiles (tile_ranges[2t]), summed from the
// masks by warp ballots.
template <int NT, int IPT_LO, int CAP, int MIN_BLOCKS, bool CHUNKED, bool ELLIPSE>
__global__ void __launch_bounds__(NT, MIN_BLOCKS)
    cell_sort_kernel(const uint32_t *__restrict__ list, const uint32_t *list_count,
                     const uint32_t *__restrict__ cell_ranges, uint64_t *words,
                     uint16_t *__restrict__ masks, uint64_t *scratch, int64_t capacity,
                     const fgs_record *__restrict__ rec, const uint32_t *__restrict__ tt,
                     int64_t n_per_view, Views vs, uint32_t *tile_ranges,
                     const unsigned long long *n_cand, uint32_t *status) {
  static_assert(NT * IPT_LO * 2 == CAP, "two word counts per class");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SegSmem<NT, CAP> &S = *reinterpret_cast<SegSmem<NT, CAP> *>(smem_raw);
  __shared__ uint32_t s_cnt[NT / 32][CELL * CELL];
  if (binning_timed_out(status) || (int64_t)*n_cand > capacity) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint64_t R = (uint64_t)n_per_view * vs.n;
  uint32_t count = *list_count;
  if (!in_bounds(count, (uint64_t)vs.total_cells + 1u, status)) count = 0u;
  for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const uint32_t c = __ldg(list + i);
    if (!in_bounds(c, (uint64_t)vs.total_cells, status)) continue;
    const uint2 rg = __ldg(reinterpret_cast<const uint2 *>(cell_ranges) + c);
    // a listed cell is never empty; bounds that a device-side error left inconsistent: skip
    if (rg.y <= rg.x || (int64_t)rg.y > capacity) {
      if (FGS_CHECK) set_status(status, ST_BOUNDS);
      continue;
    }
    const uint32_t cnt = rg.y - rg.x;
    uint64_t *cw = words + rg.x;
    uint16_t *cm = masks + rg.x;
    const View &V = vs.v[view_of_cell(vs, c)];
    const int64_t local = (int64_t)c - V.cell_offset;
    const uint32_t cy = (uint32_t)(local / V.cells_x);
    const uint32_t bx = (uint32_t)(local - (int64_t)cy * V.cells_x) * CELL, by = cy * CELL;
    uint32_t acc[CELL * CELL];
#pragma unroll
    for (int b = 0; b < CELL * CELL; ++b) acc[b] = 0u;
    if (cnt <= (uint32_t)CAP) {
      // the words with their masks, sorted in shared memory; the tile counts from the masks
      if (cnt <= (uint32_t)(NT * IPT_LO)) sort_segment<NT, IPT_LO, CAP>(S, cw, cm, cnt);
      else sort_segment<NT, 2 * IPT_LO, CAP>(S, cw, cm, cnt);
      for (uint32_t j0 = 0; j0 < cnt; j0 += NT) {
        const uint32_t j = j0 + (uint32_t)tid;
        const uint32_t m = j < cnt ? (uint32_t)S.pay[j] : 0u;
#pragma unroll
        for (int b = 0; b < CELL * CELL; ++b) acc[b] += __popc(__ballot_sync(0xffffffffu, (m >> b) & 1u));
      }
    } else if (CHUNKED) {
      // a long cell: the words sorted in chunks through the scratch buffer, then each entry's
      // mask found again from its record (plain loads: this CTA wrote the words)
      sort_segment_chunked<NT, 2 * IPT_LO, CAP>(S, cw, cnt, scratch + rg.x);
      for (uint32_t j0 = 0; j0 < cnt; j0 += NT) {
        const uint32_t j = j0 + (uint32_t)tid;
        uint32_t m = 0u;
        if (j < cnt) {
          uint32_t r = (uint32_t)cw[j];
          if (!in_bounds(r, R, status)) r = 0u;
          PairSet P;
          if (pair_set(__ldg(reinterpret_cast<const uint4 *>(rec + r) + 2), __ldg(tt + r), V, P))
            m = cell_mask(P, bx, by);
          if (ELLIPSE) m = ellipse_mask(rec + r, m, bx, by);
          cm[j] = (uint16_t)m;
        }
#pragma unroll
        for (int b = 0; b < CELL * CELL; ++b) acc[b] += __popc(__ballot_sync(0xffffffffu, (m >> b) & 1u));
      }
    } else {
      if (FGS_CHECK) set_status(status, ST_BOUNDS);  // a long cell listed in the short class
      continue;
    }
    if (lane == 0) {
#pragma unroll
      for (int b = 0; b < CELL * CELL; ++b) s_cnt[wid][b] = acc[b];
    }
    __syncthreads();
    if (tid < CELL * CELL) {
      uint32_t tot = 0;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) tot += s_cnt[w][tid];
      const uint32_t tx = bx + tid % CELL, ty = by + tid / CELL;
      if (tx < (uint32_t)V.tiles_x && ty < (uint32_t)V.tiles_y)
        tile_ranges[2 * (V.tile_offset + (int64_t)ty * V.tiles_x + tx)] = tot;
    }
    __syncthreads();
  }
}

template <int NT, int IPT_LO, int CAP, int MIN_BLOCKS, bool CHUNKED, bool ELLIPSE>
cudaError_t launch_cell_sort(const uint32_t *list, const uint32_t *list_count,
                             const uint32_t *cell_ranges, uint64_t *words, uint16_t *masks,
                             uint64_t *scratch, int64_t capacity, const fgs_record *rec,
                             const uint32_t *tt, int64_t n_per_view, const Views &vs,
                             uint32_t *tile_ranges, const unsigned long long *n_cand,
                             uint32_t *status, cudaStream_t st) {
  auto kernel = cell_sort_kernel<NT, IPT_LO, CAP, MIN_BLOCKS, CHUNKED, ELLIPSE>;
  constexpr size_t smem = sizeof(SegSmem<NT, CAP>);
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, kernel, NT, smem);
    occ = a > 0 ? a : 1;
  }
  kernel<<<(unsigned)(sm_count() * occ), NT, smem, st>>>(list, list_count, cell_ranges, words, masks,
                                                         scratch, capacity, rec, tt, n_per_view, vs,
                                                         tile_ranges, n_cand, status);
  return cudaGetLastError();
}

// Step 6. One CTA of CELL x CELL warps per cell, persistent over the cells. The cell's sorted
// list is cut into groups of 32 entries; per group, one ballot per tile bit of the masks gives
// the group's entries of each tile. (1) Every group's 16 ballots go to shared memory; (2) warp
// b scans the popcounts of tile b's ballots over the groups, from the tile's start, so each
// group knows where its entries of each tile go; (3) every group writes each of its entries
// once per tile bit, at its group's place plus its rank in the ballot. A tile's pairs thus come
// out in the cell's order, which is sorted, as key tile << 32 | depth bits and value record. A
// cell of more than EMIT_GROUPS groups is emitted one tile per warp, walking the list in order.
constexpr int CEMIT_THREADS = 32 * CELL * CELL;
constexpr int EMIT_GROUPS = 128;

__device__ __forceinline__ int64_t cell_tile(const View &V, uint32_t bx, uint32_t by, int b) {
  return V.tile_offset + (int64_t)(by + b / CELL) * V.tiles_x + bx + b % CELL;
}

// four CTAs per SM: at most 32 registers a thread
__global__ void __launch_bounds__(CEMIT_THREADS, 4)
    cell_emit_kernel(const uint32_t *__restrict__ tile_ranges,
                     const uint32_t *__restrict__ cell_ranges, const uint64_t *__restrict__ words,
                     const uint16_t *__restrict__ masks, Views vs, uint64_t *__restrict__ keys,
                     uint32_t *__restrict__ vals, int64_t capacity,
                     const unsigned long long *n_cand, uint32_t *status) {
  // per group g and tile bit b: the group's ballot of the bit and where its entries of tile b go
  __shared__ uint2 s_bp[EMIT_GROUPS][CELL * CELL];
  __shared__ uint32_t s_tile[CELL * CELL];  // global tile id of each bit
  if (binning_timed_out(status) || (int64_t)*n_cand > capacity) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t lt = lanemask_lt();
  for (int64_t c = blockIdx.x; c < vs.total_cells; c += gridDim.x) {
    const uint2 crg = __ldg(reinterpret_cast<const uint2 *>(cell_ranges) + c);
    if (crg.y <= crg.x) continue;  // uniform over the CTA
    if (!in_bounds(crg.y, (uint64_t)capacity + 1u, status) || (int64_t)crg.y > capacity) continue;
    const uint32_t cnt = crg.y - crg.x;
    const uint32_t G = (cnt + 31u) / 32u;
    const View &V = vs.v[view_of_cell(vs, c)];
    const int64_t local = c - V.cell_offset;
    const uint32_t cy = (uint32_t)(local / V.cells_x);
    const uint32_t bx = (uint32_t)(local - (int64_t)cy * V.cells_x) * CELL, by = cy * CELL;
    const uint64_t *cw = words + crg.x;
    const uint16_t *cm = masks + crg.x;
    if (G <= (uint32_t)EMIT_GROUPS) {
      __syncthreads();  // the previous cell's ballots are no longer read
      for (uint32_t g = wid; g < G; g += CELL * CELL) {  // (1)
        const uint32_t i = g * 32u + (uint32_t)lane;
        const uint32_t m = i < cnt ? (uint32_t)__ldg(cm + i) : 0u;
        uint32_t mine = 0u;
#pragma unroll
        for (int b = 0; b < CELL * CELL; ++b) {
          const uint32_t bal = __ballot_sync(0xffffffffu, (m >> b) & 1u);
          if (lane == b) mine = bal;
        }
        if (lane < CELL * CELL) s_bp[g][lane].x = mine;
      }
      __syncthreads();
      {  // (2) warp b: exclusive scan over the groups, 4 consecutive groups per lane
        const int b = wid;
        const uint32_t tx = bx + b % CELL, ty = by + b / CELL;
        uint32_t start = 0u, end = 0u;
        if (tx < (uint32_t)V.tiles_x && ty < (uint32_t)V.tiles_y) {
          const int64_t t = cell_tile(V, bx, by, b);
          const uint2 trg = __ldg(reinterpret_cast<const uint2 *>(tile_ranges) + t);
          start = trg.x;
          end = trg.y;
          if (lane == 0) s_tile[b] = (uint32_t)t;
        }
        uint32_t n4[4], sum = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t g = 4u * lane + q;
          n4[q] = g < G ? __popc(s_bp[g][b].x) : 0u;
          sum += n4[q];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        uint32_t run = start + incl - sum;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t g = 4u * lane + q;
          if (g < G) s_bp[g][b].y = run;
          run += n4[q];
        }
        // checked build: the tile receives exactly its counted pairs
        if (FGS_CHECK && lane == 31 && run != end) set_status(status, ST_BOUNDS);
      }
      __syncthreads();
      for (uint32_t g = wid; g < G; g += CELL * CELL) {  // (3)
        const uint32_t i = g * 32u + (uint32_t)lane;
        const uint64_t w = i < cnt ? __ldg(cw + i) : 0ull;
        const uint64_t kd = w >> 32;
#pragma unroll
        for (int b = 0; b < CELL * CELL; ++b) {
          const uint2 bp = s_bp[g][b];
          const uint32_t pos = bp.y + __popc(bp.x & lt);
          bool ok = (bp.x >> lane) & 1u;
          if (FGS_CHECK && ok) ok = in_bounds(pos, (uint64_t)capacity, status);
          ok = ok && (int64_t)pos < capacity;
          // predicated stores (no branch per tile bit): the address is formed for every lane
          // but only dereferenced where ok
          const uint64_t key = ((uint64_t)s_tile[b] << 32) | kd;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %3, 0;\n"
              " @p st.global.u64 [%0], %2;\n @p st.global.u32 [%1], %4;\n}"
              :: "l"(keys + pos), "l"(vals + pos), "l"(key), "r"((uint32_t)ok), "r"((uint32_t)w)
              : "memory");
        }
      }
    } else {
      // a long cell: warp w walks the list for tile w
      const uint32_t tx = bx + wid % CELL, ty = by + wid / CELL;
      if (tx < (uint32_t)V.tiles_x && ty < (uint32_t)V.tiles_y) {
        const int64_t t = cell_tile(V, bx, by, wid);
        const uint2 trg = __ldg(reinterpret_cast<const uint2 *>(tile_ranges) + t);
        if (trg.y > trg.x && in_bounds(trg.y, (uint64_t)capacity + 1u, status) &&
            (int64_t)trg.y <= capacity) {
          uint32_t o = trg.x;
          for (uint32_t g = 0; g < cnt && o < trg.y; g += 32u) {
            const uint32_t i = g + (uint32_t)lane;
            const bool kept = i < cnt && ((__ldg(cm + i) >> wid) & 1u);
            const uint32_t bal = __ballot_sync(0xffffffffu, kept);
            const uint32_t pos = o + __popc(bal & lt);
            if (kept && pos < trg.y) {
              const uint64_t w = __ldg(cw + i);
              keys[pos] = ((uint64_t)t << 32) | (w >> 32);
              vals[pos] = (uint32_t)w;
            }
            o += __popc(bal);
          }
          if (FGS_CHECK && lane == 0 && o != trg.y) set_status(status, ST_BOUNDS);
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_bin_sort(const fgs_record *records, const uint32_t *tiles_touched,
                            int64_t n, const Views &vs, uint64_t *keys, uint32_t *vals,
                            int64_t capacity, uint32_t *tile_ranges, int64_t *n_int,
                            char *ws, const WsLayout &L, uint32_t flags,
                            const CallOpts &opt, cudaStream_t st) {
  cudaError_t e;
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.header);
  uint64_t *tile_lb = reinterpret_cast<uint64_t *>(ws + L.tile_lb);
  uint64_t *cell_lb = reinterpret_cast<uint64_t *>(ws + L.cell_lb);
  uint32_t *cell_ranges = reinterpret_cast<uint32_t *>(ws + L.cell_ranges);
  uint32_t *lists = reinterpret_cast<uint32_t *>(ws + L.seg_list);
  uint64_t *words = reinterpret_cast<uint64_t *>(ws + L.words);
  uint16_t *masks = reinterpret_cast<uint16_t *>(ws + L.masks);
  const int64_t R = (int64_t)vs.n * n;
  const int64_t T = vs.total_tiles, NC = vs.total_cells;

  // the header, both look-back arrays and the cell counters are adjacent: one memset
  if ((e = cudaMemsetAsync(hdr, 0, L.g2d - L.header, st)) != cudaSuccess) return e;
  if (R == 0) {  // no pairs: every tile range empty
    if ((e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)T, st)) != cudaSuccess) return e;
    return cudaMemsetAsync(n_int, 0, sizeof(int64_t), st);
  }

  const bool ellipse = (flags & FGS_BIN_ELLIPSE) != 0;
  const unsigned rgrid = (unsigned)((R + REC_BLOCK - 1) / REC_BLOCK);
  // the per-CTA count table, when the cells fit shared memory and the table its region
  uint32_t *cta_counts = NC <= SMEM_CELLS && (int64_t)rgrid * NC <= L.cell_count_entries
                             ? reinterpret_cast<uint32_t *>(ws + L.cell_counts) : nullptr;
  cell_count_kernel<<<rgrid, REC_THREADS, 0, st>>>(records, tiles_touched, R, n, vs, capacity,
                                                   cell_ranges, cta_counts, &hdr->n_candidates,
                                                   &hdr->n_visible, &hdr->status);
  tile_scan_kernel<false><<<(unsigned)((NC + TSCAN_PART - 1) / TSCAN_PART), 256, 0, st>>>(
      cell_ranges, NC, cell_lb, &hdr->cell_parts, lists, hdr->seg_count, (uint32_t)CELL_CAP0,
      &hdr->n_candidates, capacity, nullptr, &hdr->status, opt.wait_limit, vs, nullptr);
  if (ellipse)
    cell_scatter_kernel<true><<<rgrid, REC_THREADS, 0, st>>>(
        records, tiles_touched, R, n, vs, cell_ranges, words, masks, cta_counts,
        &hdr->n_candidates, capacity, &hdr->status);
  else
    cell_scatter_kernel<false><<<rgrid, REC_THREADS, 0, st>>>(
        records, tiles_touched, R, n, vs, cell_ranges, words, masks, cta_counts,
        &hdr->n_candidates, capacity, &hdr->status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the keys output serves as the chunked sort's scratch (it is written only by the last step)
  if (ellipse) {
    if ((e = launch_cell_sort<512, 4, CELL_CAP0, 2, false, true>(
             lists, &hdr->seg_count[0], cell_ranges, words, masks, keys, capacity, records,
             tiles_touched, n, vs, tile_ranges, &hdr->n_candidates, &hdr->status, st)) != cudaSuccess)
      return e;
    if ((e = launch_cell_sort<512, 8, SEG_CAP1, 1, true, true>(
             lists + NC, &hdr->seg_count[1], cell_ranges, words, masks, keys, capacity, records,
             tiles_touched, n, vs, tile_ranges, &hdr->n_candidates, &hdr->status, st)) != cudaSuccess)
      return e;
  } else {
    if ((e = launch_cell_sort<512, 4, CELL_CAP0, 2, false, false>(
             lists, &hdr->seg_count[0], cell_ranges, words, masks, keys, capacity, records,
             tiles_touched, n, vs, tile_ranges, &hdr->n_candidates, &hdr->status, st)) != cudaSuccess)
      return e;
    if ((e = launch_cell_sort<512, 8, SEG_CAP1, 1, true, false>(
             lists + NC, &hdr->seg_count[1], cell_ranges, words, masks, keys, capacity, records,
             tiles_touched, n, vs, tile_ranges, &hdr->n_candidates, &hdr->status, st)) != cudaSuccess)
      return e;
  }
  tile_scan_kernel<true><<<(unsigned)L.tile_parts, 256, 0, st>>>(
      tile_ranges, T, tile_lb, &hdr->tile_parts, nullptr, nullptr, 0u, &hdr->n_candidates,
      capacity, n_int, &hdr->status, opt.wait_limit, vs, cell_ranges);
  static int eocc = 0;
  if (eocc == 0) {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cell_emit_kernel, CEMIT_THREADS, 0);
    eocc = a > 0 ? a : 1;
  }
  int64_t egrid = (int64_t)sm_count() * eocc;
  if (egrid > NC) egrid = NC;
  cell_emit_kernel<<<(unsigned)(egrid > 0 ? egrid : 1), CEMIT_THREADS, 0, st>>>(
      tile_ranges, cell_ranges, words, masks, vs, keys, vals, capacity, &hdr->n_candidates,
      &hdr->status);
  return cudaGetLastError();
}

}  // namespace fgs
