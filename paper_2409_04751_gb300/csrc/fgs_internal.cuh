// fgs_internal.cuh - shared device code of the fisheye Gaussian-splatting kernels (sm_103a).
//
// Everything here is written from the method's mathematics (Fisheye-GS, arXiv 2409.04751):
// the equidistant projection (Sec. 3.2), its Jacobian (Sec. 4.2, with f on the theta terms)
// and the derivative of the Jacobian (Sec. 4.3), in a form that stays accurate near the
// optical axis.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fgs.h"

namespace fgs {

// ------------------------------------------------------------------------------------------
// Renderer conventions (the paper inherits them from the 3DGS rasteriser and fixes none):
constexpr int TILE = FGS_TILE;
constexpr float NEAR_DIST = 0.2f;                         // cull |mu_c| <= 0.2
constexpr float THETA_MAX = 3.14159265358979f - 0.05f;    // cull the singular cone theta -> pi
constexpr float ALPHA_MIN = 1.0f / 255.0f;                // contribution threshold
constexpr float ALPHA_MAX = 0.99f;                        // alpha cap
constexpr float T_MIN = 1e-4f;                            // transmittance stop
constexpr float DILATION = 0.3f;                          // added to Sigma_p's diagonal
constexpr float LOG2E = 1.4426950408889634f;
constexpr float LOG2_ALPHA_MIN = -7.994353436858858f;     // log2(1/255)
constexpr float SERIES_T = 0.3f;                          // near-axis series below t = l_z/z

// Device status codes (same values as fgs_status).
constexpr uint32_t ST_CAPACITY = FGS_ERR_CAPACITY;
constexpr uint32_t ST_TIMEOUT = FGS_ERR_TIMEOUT;
constexpr uint32_t ST_BOUNDS = FGS_ERR_BOUNDS;

// Checked build: -DFGS_CHECK=1 compiles the index checks of in_bounds() in (libfgs_check.so);
// the product build leaves them out.
#ifndef FGS_CHECK
#define FGS_CHECK 0
#endif

// Bounded waits: polls before a wait gives up and reports FGS_ERR_TIMEOUT. A 48-byte bulk copy
// lands within microseconds and a look-back predecessor publishes within one partition's work,
// so these limits (about a second of polling) are only reached if something is broken. The
// look-back waits take their limit per call (fgs_options.wait_limit; 0 = give up at once).
constexpr uint32_t SPIN_LIMIT = 1u << 20;

// Options of one call, resolved from fgs_options (api.cu).
struct CallOpts {
  int fwd_ppt = 4;                   // pixels per thread of the forward rasterizer (1, 2, 4)
  int bwd_ppt = 8;                   // of the backward rasterizer (1, 2, 4, 8)
  bool instrument = false;           // count work into the workspace counters
  uint32_t wait_limit = SPIN_LIMIT;  // polls of a look-back wait before it gives up
  cudaEvent_t ev_before = nullptr;   // recorded around the call's main kernel (a measurement
  cudaEvent_t ev_after = nullptr;    // hook; both or neither)
};

// ------------------------------------------------------------------------------------------
// Per-view parameters, passed by value in the kernel parameter space (no device copy).
struct View {
  float W[9];
  float b[3];
  float fx, fy, cx, cy;
  float cam_pos[3];  // camera centre -W^T b
  int32_t width, height, tiles_x, tiles_y;
  int32_t model;     // fgs_camera_model
  int32_t cells_x;   // binning cells (CELL x CELL tiles) per row of the view
  int64_t tile_offset, pixel_offset;
  int64_t cell_offset;  // first global cell id of the view
};

struct Views {
  int32_t n;
  int32_t tile_bits;
  int64_t total_tiles, total_pixels, total_cells;
  View v[FGS_MAX_VIEWS];
};

// The binning groups tiles into cells of CELL x CELL tiles (view-major, row-major inside a
// view, the last row and column of a view ragged).
constexpr int CELL = 4;

// global tile -> view (views are few; binary search over the tile offsets)
__device__ __forceinline__ int view_of_tile(const Views &vs, int64_t t) {
  int lo = 0, hi = vs.n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (vs.v[mid].tile_offset <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// global cell -> view
__device__ __forceinline__ int view_of_cell(const Views &vs, int64_t c) {
  int lo = 0, hi = vs.n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (vs.v[mid].cell_offset <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------------------------------
// Workspace layout (bytes from the workspace base; every region 256-byte aligned).
struct WsHeader {
  uint32_t status;            // fgs_status of device-detected errors (first one wins)
  uint32_t scan_parts;        // partition counter of the tiles_touched scan
  uint32_t tile_parts;        // partition counter of the per-tile count scan
  uint32_t seg_count[2];      // cells in each segment-size class (filled by the cell scan)
  uint32_t cell_parts;        // partition counter of the per-cell count scan
  uint32_t spare[4];
  uint32_t raster_tiles;      // tile queue of the forward rasterizer
  uint32_t spare2;            // (the backward's tile queue sits with its tile order)
  // measurement counters, written only by instrumented launches (FGS_OPT_INSTRUMENT):
  // [0] forward (pixel, Gaussian) evaluations, [1] forward blends,
  // [2] backward evaluations, [3] backward contributions,
  // [4] records the forward staged (copied into shared memory), [5] the backward's
  unsigned long long counters[6];
  unsigned long long n_visible;  // records with a non-empty rect (written by the scan)
  unsigned long long n_candidates;  // (record, tile) pairs of the rects (written by the scan)
  unsigned long long n_dropped;  // onesweep emission: pairs beyond their record's rect
  // checked build only, written by the binning for the rasterizers' index checks:
  uint32_t bounds_magic;         // BOUNDS_MAGIC once a binning on this workspace set the two
  uint32_t bounds_records;       // records of that binning (list entries must be below)
  uint32_t bounds_pairs;         // its key capacity (list ends must not exceed it)
  uint32_t pad[31];
};
static_assert(sizeof(WsHeader) == 256, "header size");
static_assert(offsetof(WsHeader, status) == 0, "the status word starts the header");
constexpr uint32_t BOUNDS_MAGIC = 0x4b434746u;

constexpr int EMIT_THREADS = 256;
constexpr int EMIT_ITEMS = 16;
constexpr int EMIT_PART = EMIT_THREADS * EMIT_ITEMS;  // records per scan partition
constexpr int EMIT_CHUNK = 1024;                      // (record, tile) pairs per emission CTA
constexpr int TSCAN_PART = 1024;                     // tiles per partition of the tile scan
constexpr int WORK_BUCKETS = 32;                     // log2 classes of a tile's backward work
// device-wide onesweep radix sort (onesweep.cu)
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_PART = SORT_THREADS * SORT_ITEMS;  // keys per sort partition
constexpr int SORT_MAX_PASSES = 8;
// Segment-size classes of the per-tile sort: segments of at most SEG_CAP0 pairs are sorted
// in shared memory by CTAs of 256 threads, longer ones by CTAs of 512 threads (in shared memory
// up to SEG_CAP1 pairs, beyond that in SEG_CAP1-pair chunks through global memory).
constexpr int SEG_CAP0 = 1024;
constexpr int SEG_CAP1 = 8192;
constexpr int G2D_STRIDE = 12;                        // floats per record of screen-space grads
// the cell walks of the binning (binsort.cu): records per CTA, cell counters a CTA holds in
// shared memory, and the bound of the per-CTA count table
constexpr int CELL_WALK_BLOCK = 1024;
constexpr int CELL_WALK_SMEM = 4096;
constexpr int64_t CELL_COUNTS_MAX = (int64_t)1 << 22;

struct WsLayout {
  size_t header, scan_lb, tile_lb, cell_lb, cell_ranges, g2d, tile_order, vis_rec, vis_off,
      seg_list, words, masks, chunk_first, cell_counts;
  size_t sort_hist, sort_lb, alt_vals;  // the onesweep sort's regions (0 bytes unless requested)
  size_t total;
  int64_t scan_parts, tile_parts, chunks, total_tiles, sort_parts;
  int64_t cell_count_entries;  // capacity of cell_counts (per-CTA cell counts of the cell walk)
};

__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout. Regions that depend on the record and tile counts only come first, so the
// backward can locate them without knowing the key capacity (the forward rasterizer uses the
// header alone); with_g2d = false leaves out the backward's accumulator (used by the sort-only
// variant);
// with_onesweep adds the regions of the device-wide radix sort (onesweep.cu).
constexpr WsLayout ws_layout_ex(int64_t n_records, int64_t capacity, int64_t total_tiles,
                                bool with_g2d, bool with_onesweep = false) {
  WsLayout L{};
  const int64_t R = n_records > 0 ? n_records : 1;
  const int64_t T = total_tiles > 0 ? total_tiles : 1;
  L.scan_parts = (n_records + EMIT_PART - 1) / EMIT_PART;
  L.tile_parts = (T + TSCAN_PART - 1) / TSCAN_PART;
  L.chunks = (capacity + EMIT_CHUNK - 1) / EMIT_CHUNK;
  L.total_tiles = T;
  size_t o = 0;
  // header, the look-back arrays and the per-cell counters first: one memset clears them (a
  // view has at most as many cells as tiles, so tile counts bound the cell regions)
  L.header = o; o += align256(256);
  L.scan_lb = o; o += align256(sizeof(uint64_t) * 2 * (size_t)(L.scan_parts > 0 ? L.scan_parts : 1));
  L.tile_lb = o; o += align256(sizeof(uint64_t) * (size_t)L.tile_parts);
  L.cell_lb = o; o += align256(sizeof(uint64_t) * (size_t)L.tile_parts);
  L.cell_ranges = o; o += align256(sizeof(uint32_t) * 2 * (size_t)T);
  L.g2d = o; if (with_g2d) o += align256(sizeof(float) * G2D_STRIDE * (size_t)R);
  // the backward's tile order: per-tile work bucket, tile ids by decreasing work, histogram
  L.tile_order = o; if (with_g2d) o += align256(sizeof(uint32_t) * (2 * (size_t)T + 2 * WORK_BUCKETS + 1));
  L.vis_rec = o; o += align256(sizeof(uint32_t) * (size_t)R);
  L.vis_off = o; o += align256(sizeof(uint64_t) * (size_t)R);
  L.seg_list = o; o += align256(sizeof(uint32_t) * 2 * (size_t)T);
  // cell entries (depth bits << 32 | record) and their tile masks; 4 entries of slack so that
  // groups of 4 read from a multiple of 4 stay inside
  L.words = o; o += align256(sizeof(uint64_t) * ((size_t)capacity + 4));
  L.masks = o; o += align256(sizeof(uint16_t) * ((size_t)capacity + 4));
  L.chunk_first = o; o += align256(sizeof(uint32_t) * ((size_t)L.chunks + 2));
  // each cell-walk CTA's counts per cell, kept for the scatter when they fit (views of at most
  // CELL_WALK_SMEM cells; at most CELL_COUNTS_MAX entries)
  {
    const int64_t blocks = (n_records + CELL_WALK_BLOCK - 1) / CELL_WALK_BLOCK;
    const int64_t cells = T < CELL_WALK_SMEM ? T : CELL_WALK_SMEM;
    const int64_t want = blocks * cells;
    L.cell_count_entries = want < CELL_COUNTS_MAX ? want : CELL_COUNTS_MAX;
  }
  L.cell_counts = o; o += align256(sizeof(uint32_t) * (size_t)(L.cell_count_entries + 1));
  L.sort_parts = (capacity + SORT_PART - 1) / SORT_PART;
  L.sort_hist = o;
  if (with_onesweep) o += align256(sizeof(uint32_t) * SORT_MAX_PASSES * 256);
  L.sort_lb = o;
  if (with_onesweep)
    o += align256(sizeof(uint64_t) * 256 * 2 * (size_t)(L.sort_parts > 0 ? L.sort_parts : 1));
  L.alt_vals = o;
  if (with_onesweep) o += align256(sizeof(uint32_t) * ((size_t)capacity + 4));
  L.total = o;
  return L;
}

inline WsLayout ws_layout(int64_t n_records, int64_t capacity, int64_t total_tiles,
                          bool with_onesweep = false) {
  return ws_layout_ex(n_records, capacity, total_tiles, true, with_onesweep);
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t code) {
  atomicCAS(status, 0u, code);
}

// Index check of the checked build: true if i < n; otherwise FGS_ERR_BOUNDS is recorded and
// the caller skips the access. Always true (and compiled away) in the product build.
__device__ __forceinline__ bool in_bounds(uint64_t i, uint64_t n, uint32_t *status) {
  if (!FGS_CHECK || i < n) return true;
  set_status(status, ST_BOUNDS);
  return false;
}

// Bounds of the rasterizers' index checks: the record count and key capacity recorded by the
// binning on this workspace (the status word starts the header), or no bound when none did.
struct ListBounds {
  uint32_t records, pairs;
};
__device__ __forceinline__ ListBounds list_bounds(const uint32_t *status) {
  ListBounds b{0xffffffffu, 0xffffffffu};
  if (FGS_CHECK) {
    const WsHeader *h = reinterpret_cast<const WsHeader *>(status);
    if (h->bounds_magic == BOUNDS_MAGIC) b = ListBounds{h->bounds_records, h->bounds_pairs};
  }
  return b;
}

// A look-back wait of an earlier kernel of the same binning gave up: its offsets are partial,
// so the kernels after it leave their outputs alone (the status word keeps the error).
__device__ __forceinline__ bool binning_timed_out(const uint32_t *status) {
  return *(volatile const uint32_t *)status == ST_TIMEOUT;
}

// ------------------------------------------------------------------------------------------
// PTX helpers: mbarrier + TMA bulk copy (cp.async.bulk), sm_90+ forms used on sm_103a.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; returns false (and records FGS_ERR_TIMEOUT) on give-up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t *status) {
  for (uint32_t it = 0; it < SPIN_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  set_status(status, ST_TIMEOUT);
  return false;
}

// One TMA bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-aligned),
// completing `bytes` transactions on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Hardware approximations (single MUFU instructions): 2^x with relative error below 2^-22 and
// 1/x with relative error below 2^-23, subnormals flushed. The blend's alpha >= 1/255 and the
// transmittance >= 1e-4 never reach the subnormal range.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_volatile_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------------------------------------------------------
// Equidistant projection pieces. With u = l_z = |(x, y)|, l2 = |mu_c|^2, theta = atan2(u, z):
//   g   = theta / u                       (x_p = cx + fx g x, y_p = cy + fy g y)
//   h   = dg/du / u = (z u / l2 - theta) / u^3
//   huu = dh/du / u = -(2 z / l2^2 + 3 h) / u^2
// so that J = [[fx (g + x^2 h), fx x y h, -fx x / l2], [fy x y h, fy (g + y^2 h), -fy y / l2]].
// Near the axis (0 < t = u / z < SERIES_T) h and huu cancel catastrophically; there the
// Taylor series in t (from atan t = sum (-1)^k t^(2k+1) / (2k+1)) are used:
//   g   = z^-1 sum_{k>=0} (-1)^k t^2k / (2k+1)
//   h   = z^-3 sum_{k>=1} (-1)^k 2k/(2k+1) t^(2k-2)
//   huu = z^-5 sum_{k>=2} (-1)^k 2k (2k-2)/(2k+1) t^(2k-4)
struct FishG {
  float theta, g, h, huu;
};

template <bool NEED_HUU>
__device__ __forceinline__ FishG fisheye_g(float x, float y, float z) {
  FishG r;
  float u2 = x * x + y * y;
  float u = sqrtf(u2);
  float l2 = u2 + z * z;
  r.theta = atan2f(u, z);
  if (z > 0.f && u < SERIES_T * z) {
    float iz = 1.0f / z;
    float t2 = u2 * iz * iz;
    // Horner in t2; coefficients (-1)^k / (2k+1), k = 0..9
    float sg = -1.f / 19.f;
    sg = fmaf(sg, t2, 1.f / 17.f); sg = fmaf(sg, t2, -1.f / 15.f); sg = fmaf(sg, t2, 1.f / 13.f);
    sg = fmaf(sg, t2, -1.f / 11.f); sg = fmaf(sg, t2, 1.f / 9.f); sg = fmaf(sg, t2, -1.f / 7.f);
    sg = fmaf(sg, t2, 1.f / 5.f); sg = fmaf(sg, t2, -1.f / 3.f); sg = fmaf(sg, t2, 1.f);
    // (-1)^k 2k/(2k+1), k = 1..9
    float sh = -18.f / 19.f;
    sh = fmaf(sh, t2, 16.f / 17.f); sh = fmaf(sh, t2, -14.f / 15.f); sh = fmaf(sh, t2, 12.f / 13.f);
    sh = fmaf(sh, t2, -10.f / 11.f); sh = fmaf(sh, t2, 8.f / 9.f); sh = fmaf(sh, t2, -6.f / 7.f);
    sh = fmaf(sh, t2, 4.f / 5.f); sh = fmaf(sh, t2, -2.f / 3.f);
    float iz3 = iz * iz * iz;
    r.g = sg * iz;
    r.h = sh * iz3;
    if (NEED_HUU) {
      // (-1)^k 2k(2k-2)/(2k+1), k = 2..10
      float s8 = 360.f / 21.f;
      s8 = fmaf(s8, t2, -288.f / 19.f); s8 = fmaf(s8, t2, 224.f / 17.f);
      s8 = fmaf(s8, t2, -168.f / 15.f); s8 = fmaf(s8, t2, 120.f / 13.f);
      s8 = fmaf(s8, t2, -80.f / 11.f); s8 = fmaf(s8, t2, 48.f / 9.f);
      s8 = fmaf(s8, t2, -24.f / 7.f); s8 = fmaf(s8, t2, 8.f / 5.f);
      r.huu = s8 * iz3 * iz * iz;
    } else {
      r.huu = 0.f;
    }
  } else {
    r.g = r.theta / u;
    r.h = (z * u / l2 - r.theta) / (u2 * u);
    r.huu = NEED_HUU ? -(2.f * z / (l2 * l2) + 3.f * r.h) / u2 : 0.f;
  }
  return r;
}

// ------------------------------------------------------------------------------------------
// Ellipse-tile test of the binning's exact mode. A Gaussian can reach alpha >= 1/255 at a pixel
// of a tile only if the minimum over the tile's rectangle of pixel centres [xl, xh] x [yl, yh]
// of q(d) = A dx^2 + 2 B dx dy + C dy^2 (conic (A, B, C), d = pixel - mean) is at most
// q* = 2 ln(255 opacity). The minimum of this convex quadratic over the rectangle is 0 with the
// mean inside it, else it lies on an edge, where it is the 1D minimum in the free coordinate
// clamped to the edge. The pair is kept when the minimum is at most q* (1 + 1e-3) + 1e-2, a
// margin far above the rounding of the rasterizer's exponent, so no contributing pair is lost.
// The per-Gaussian part (threshold and the two reciprocals) is computed once and reused for
// every tile the Gaussian's rect covers.
struct EllipseTest {
  float mx, my, A, B, C, thr, iA, iC;
};

__device__ __forceinline__ EllipseTest ellipse_test(float mx, float my, float A, float B, float C,
                                                    float qs) {
  EllipseTest E;
  E.mx = mx; E.my = my; E.A = A; E.B = B; E.C = C;
  E.thr = fmaf(qs, 1.001f, 1e-2f);
  E.iA = 1.f / A;
  E.iC = 1.f / C;
  return E;
}

__device__ __forceinline__ bool ellipse_reaches_tile(const EllipseTest &E, float xl, float xh,
                                                     float yl, float yh) {
  const float mx = E.mx, my = E.my, A = E.A, B = E.B, C = E.C;
  if (mx >= xl && mx <= xh && my >= yl && my <= yh) return true;
  float qmin = 3.0e38f;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    // vertical edge x = xl or xh: dy* = -B dx / C, clamped
    const float dx = (e ? xh : xl) - mx;
    const float dy = fminf(fmaxf(-B * dx * E.iC, yl - my), yh - my);
    qmin = fminf(qmin, fmaf(dx, fmaf(A, dx, 2.f * B * dy), C * dy * dy));
    // horizontal edge y = yl or yh: dx* = -B dy / A, clamped
    const float ey = (e ? yh : yl) - my;
    const float ex = fminf(fmaxf(-B * ey * E.iA, xl - mx), xh - mx);
    qmin = fminf(qmin, fmaf(ex, fmaf(A, ex, 2.f * B * ey), C * ey * ey));
  }
  return qmin <= E.thr;
}

// ------------------------------------------------------------------------------------------
// Every camera model: field of view, projection of the mean, Jacobian J (2x3) and, for the
// backward, dL/dmu_c from dL/dJ.
//
// Radial models (x_p = cx + fx g x, y_p = cy + fy g y, g = r(theta) / l_z a function G(l, z) of
// l = |mu_c| and z) share one Jacobian,
//   J = [[fx (g + x^2 h), fx x y h, fx x k], [fy x y h, fy (g + y^2 h), fy y k]],
// h = G_l / l, k = G_z + z h (so dg/dx = x h, dg/dz = k). The backward also needs
// h_l, k_l = (1/l) d/dl at fixed z (dh/dx = x h_l, dk/dx = x k_l) and h_z, k_z = d/dz at fixed
// x, y. Equidistant: g, h, h_l from fisheye_g, k = -1/l2, h_z = k_l = 2/l2^2, k_z = 2 z/l2^2.
// The others from closed forms of G (cos theta = z / l):
//   equisolid      G = sqrt(2 / (l (l + z)))
//   stereographic  G = 2 / (l + z)
//   orthographic   G = 1 / l
//   pinhole        G = 1 / z
constexpr float COS_THETA_MAX = -0.99875026039f;       // cos(pi - 0.05)
constexpr float COS_THETA_MAX_ORTHO = 0.04997916927f;  // cos(pi/2 - 0.05)
constexpr float SIN_LAT_MAX = 0.99875026039f;          // sin(pi/2 - 0.05)

struct RadTerms {
  float g, h, k, hl, hz, kl, kz;
};

template <bool BWD>
__device__ __forceinline__ RadTerms radial_terms(int model, float x, float y, float z, float l2) {
  RadTerms t;
  const float il2 = 1.f / l2;
  if (model == FGS_CAM_EQUIDISTANT) {
    const FishG fg = fisheye_g<BWD>(x, y, z);
    t.g = fg.g;
    t.h = fg.h;
    t.k = -il2;
    t.hl = fg.huu;
    t.hz = 2.f * il2 * il2;
    t.kl = t.hz;
    t.kz = z * t.hz;
    return t;
  }
  const float l = sqrtf(l2), il = 1.f / l;
  // l + z, without the cancellation of z ~ -l behind the camera: (x^2 + y^2) / (l - z) there
  const float lpz = z >= 0.f ? l + z : (x * x + y * y) / (l - z);
  float G0, G1, G2, G3, G4, G5;  // G, G_l, G_z, G_ll, G_lz, G_zz
  if (model == FGS_CAM_EQUISOLID) {
    const float P = l * lpz, Pl = l + lpz, Pz = l;
    const float Pm12 = rsqrtf(P), Pm32 = Pm12 / P, Pm52 = Pm32 / P;
    const float r2 = 1.41421356237f;
    G0 = r2 * Pm12;
    G1 = -0.5f * r2 * Pm32 * Pl;
    G2 = -0.5f * r2 * Pm32 * Pz;
    G3 = 0.75f * r2 * Pm52 * Pl * Pl - r2 * Pm32;
    G4 = 0.75f * r2 * Pm52 * Pl * Pz - 0.5f * r2 * Pm32;
    G5 = 0.75f * r2 * Pm52 * Pz * Pz;
  } else if (model == FGS_CAM_STEREOGRAPHIC) {
    const float iS = 1.f / lpz;
    G0 = 2.f * iS;
    G1 = G2 = -2.f * iS * iS;
    G3 = G4 = G5 = 4.f * iS * iS * iS;
  } else if (model == FGS_CAM_PINHOLE) {  // g = 1 / z
    const float iz = 1.f / z;
    G0 = iz;
    G1 = 0.f;
    G2 = -iz * iz;
    G3 = G4 = 0.f;
    G5 = 2.f * iz * iz * iz;
  } else {  // orthographic
    G0 = il;
    G1 = -il * il;
    G2 = 0.f;
    G3 = 2.f * il * il * il;
    G4 = G5 = 0.f;
  }
  t.g = G0;
  t.h = G1 * il;
  t.k = fmaf(z, t.h, G2);
  if (BWD) {
    const float Hl = (G3 - G1 * il) * il, Hz = G4 * il;
    const float Kl = fmaf(z, Hl, G4), Kz = G5 + t.h + z * Hz;
    t.hl = Hl * il;
    t.hz = fmaf(z, t.hl, Hz);
    t.kl = Kl * il;
    t.kz = fmaf(z, t.kl, Kz);
  } else {
    t.hl = t.hz = t.kl = t.kz = 0.f;
  }
  return t;
}

// Inside the model's field of view (the angle tests of the readings, written without atan2
// for the closed-form models: theta < theta_max <=> z > l cos(theta_max), and for the panorama
// |latitude| < pi/2 - 0.05 <=> |y| < l sin(pi/2 - 0.05)).
__device__ __forceinline__ bool in_field(int model, float x, float y, float z, float dist) {
  if (model == FGS_CAM_EQUIRECTANGULAR) return fabsf(y) < SIN_LAT_MAX * dist;
  if (model == FGS_CAM_EQUIDISTANT) return atan2f(sqrtf(x * x + y * y), z) < THETA_MAX;
  if (model == FGS_CAM_ORTHOGRAPHIC || model == FGS_CAM_PINHOLE) return z > COS_THETA_MAX_ORTHO * dist;
  return z > COS_THETA_MAX * dist;
}

// The pinhole camera's guard band: its projected mean within 1.3 times the half image of the
// principal point (the 1.3 tan(FOV/2) limit of the pinhole renderer the method is compared
// with, applied as a cull; beyond it a Gaussian reaches the image only with the tail of an
// ill-conditioned affine footprint).
constexpr float PINHOLE_GUARD_HALF = 0.65f;  // 1.3 / 2
__device__ __forceinline__ bool in_pinhole_guard(const View &V, float px, float py) {
  return fabsf(px - V.cx) <= PINHOLE_GUARD_HALF * (float)V.width &&
         fabsf(py - V.cy) <= PINHOLE_GUARD_HALF * (float)V.height;
}

// Projection of the mean and J (row-major 2x3) of view V at mu_c.
__device__ __forceinline__ void project_mean(const View &V, float x, float y, float z, float l2,
                                             float &px, float &py, float (&J)[6]) {
  if (V.model == FGS_CAM_EQUIRECTANGULAR) {
    // Sec. 6: x_p = cx + fx atan2(x, z), y_p = cy + fy atan2(y, rho), rho = sqrt(x^2 + z^2)
    const float r2 = x * x + z * z, rho = sqrtf(r2), ir2 = 1.f / r2, u = 1.f / (rho * l2);
    px = fmaf(V.fx, atan2f(x, z), V.cx);
    py = fmaf(V.fy, atan2f(y, rho), V.cy);
    J[0] = V.fx * z * ir2; J[1] = 0.f; J[2] = -V.fx * x * ir2;
    J[3] = -V.fy * x * y * u; J[4] = V.fy * rho / l2; J[5] = -V.fy * y * z * u;
    return;
  }
  const RadTerms t = radial_terms<false>(V.model, x, y, z, l2);
  px = fmaf(V.fx * t.g, x, V.cx);
  py = fmaf(V.fy * t.g, y, V.cy);
  J[0] = V.fx * fmaf(x * x, t.h, t.g); J[1] = V.fx * x * y * t.h; J[2] = V.fx * x * t.k;
  J[3] = V.fy * x * y * t.h; J[4] = V.fy * fmaf(y * y, t.h, t.g); J[5] = V.fy * y * t.k;
}

// dL/dmu_c through J (Sec. 4.3 for the equidistant model), from dL/dJ (row-major 2x3).
// Radial models: with A..F the f-scaled dL/dJ entries, the J-dependent part of L is
//   (A + E) g + Q h + P k,  Q = A x^2 + (B + D) x y + E y^2,  P = C x + F y.
__device__ __forceinline__ void jacobian_backward(const View &V, float x, float y, float z,
                                                  float l2, const float (&GJ)[6],
                                                  float &d0, float &d1, float &d2) {
  const float A = V.fx * GJ[0], B = V.fx * GJ[1], Cc = V.fx * GJ[2];
  const float Dd = V.fy * GJ[3], E = V.fy * GJ[4], F = V.fy * GJ[5];
  if (V.model == FGS_CAM_EQUIRECTANGULAR) {
    // J = [[fx z/rho^2, 0, -fx x/rho^2], [-fy x y u, fy rho/l2, -fy y z u]], u = 1/(rho l2):
    // du/dx = -x u w, du/dz = -z u w (w = 1/rho^2 + 2/l2), du/dy = -2 y u / l2
    const float r2 = x * x + z * z, rho = sqrtf(r2), ir2 = 1.f / r2, ir4 = ir2 * ir2;
    const float u = 1.f / (rho * l2), il2 = 1.f / l2, w = ir2 + 2.f * il2;
    const float q = u - 2.f * rho * il2 * il2;
    d0 = A * (-2.f * x * z * ir4) + Cc * (x * x - z * z) * ir4 + Dd * y * u * (x * x * w - 1.f) +
         E * x * q + F * x * y * z * u * w;
    d1 = Dd * x * u * (2.f * y * y * il2 - 1.f) - E * 2.f * y * rho * il2 * il2 +
         F * z * u * (2.f * y * y * il2 - 1.f);
    d2 = A * (x * x - z * z) * ir4 + Cc * 2.f * x * z * ir4 + Dd * x * y * z * u * w + E * z * q +
         F * y * u * (z * z * w - 1.f);
    return;
  }
  (void)B;
  const RadTerms t = radial_terms<true>(V.model, x, y, z, l2);
  const float AE = A + E, BD = B + Dd;
  const float Q = A * x * x + BD * x * y + E * y * y;
  const float P = Cc * x + F * y;
  d0 = AE * x * t.h + (2.f * A * x + BD * y) * t.h + Q * t.hl * x + Cc * t.k + P * x * t.kl;
  d1 = AE * y * t.h + (BD * x + 2.f * E * y) * t.h + Q * t.hl * y + F * t.k + P * y * t.kl;
  d2 = AE * t.k + Q * t.hz + P * t.kz;
}

// ------------------------------------------------------------------------------------------
// Real spherical harmonics up to degree 3 (Condon-Shortley phase, order m = -l..l) as
// polynomials of the unit direction (x, y, z). Constants are the normalisations
//   c0 = 1/(2 sqrt(pi)); c1 = sqrt(3/(4 pi));
//   c2a = sqrt(15/pi)/2, c2b = sqrt(5/pi)/4, c2c = sqrt(15/pi)/4;
//   c3a = sqrt(35/(2 pi))/4, c3b = sqrt(105/pi)/2, c3c = sqrt(21/(2 pi))/4,
//   c3d = sqrt(7/pi)/4, c3e = sqrt(105/pi)/4.
constexpr float SH_C0 = 0.28209479177387814f;
constexpr float SH_C1 = 0.48860251190291992f;
constexpr float SH_C2A = 1.0925484305920792f;
constexpr float SH_C2B = 0.31539156525252005f;
constexpr float SH_C2C = 0.54627421529603959f;
constexpr float SH_C3A = 0.59004358992664352f;
constexpr float SH_C3B = 2.8906114426405538f;
constexpr float SH_C3C = 0.45704579946446572f;
constexpr float SH_C3D = 0.37317633259011540f;
constexpr float SH_C3E = 1.4453057213202769f;

template <int D>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
  Y[0] = SH_C0;
  if (D >= 1) {
    Y[1] = -SH_C1 * y; Y[2] = SH_C1 * z; Y[3] = -SH_C1 * x;
  }
  if (D >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH_C2A * x * y;
    Y[5] = -SH_C2A * y * z;
    Y[6] = SH_C2B * (2.f * zz - xx - yy);
    Y[7] = -SH_C2A * x * z;
    Y[8] = SH_C2C * (xx - yy);
    if (D >= 3) {
      Y[9] = -SH_C3A * y * (3.f * xx - yy);
      Y[10] = SH_C3B * x * y * z;
      Y[11] = -SH_C3C * y * (4.f * zz - xx - yy);
      Y[12] = SH_C3D * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -SH_C3C * x * (4.f * zz - xx - yy);
      Y[14] = SH_C3E * z * (xx - yy);
      Y[15] = -SH_C3A * x * (xx - 3.f * yy);
    }
  }
}

// d Y_k / d(x, y, z) of the polynomials above (their tangential part is the derivative on
// the sphere, which is all the backward uses).
template <int D>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float (*dY)[3]) {
  dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
  if (D >= 1) {
    dY[1][0] = 0.f; dY[1][1] = -SH_C1; dY[1][2] = 0.f;
    dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = SH_C1;
    dY[3][0] = -SH_C1; dY[3][1] = 0.f; dY[3][2] = 0.f;
  }
  if (D >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    dY[4][0] = SH_C2A * y; dY[4][1] = SH_C2A * x; dY[4][2] = 0.f;
    dY[5][0] = 0.f; dY[5][1] = -SH_C2A * z; dY[5][2] = -SH_C2A * y;
    dY[6][0] = -2.f * SH_C2B * x; dY[6][1] = -2.f * SH_C2B * y; dY[6][2] = 4.f * SH_C2B * z;
    dY[7][0] = -SH_C2A * z; dY[7][1] = 0.f; dY[7][2] = -SH_C2A * x;
    dY[8][0] = 2.f * SH_C2C * x; dY[8][1] = -2.f * SH_C2C * y; dY[8][2] = 0.f;
    if (D >= 3) {
      dY[9][0] = -6.f * SH_C3A * x * y; dY[9][1] = -SH_C3A * (3.f * xx - 3.f * yy); dY[9][2] = 0.f;
      dY[10][0] = SH_C3B * y * z; dY[10][1] = SH_C3B * x * z; dY[10][2] = SH_C3B * x * y;
      dY[11][0] = 2.f * SH_C3C * x * y; dY[11][1] = -SH_C3C * (4.f * zz - xx - 3.f * yy);
      dY[11][2] = -8.f * SH_C3C * y * z;
      dY[12][0] = -6.f * SH_C3D * x * z; dY[12][1] = -6.f * SH_C3D * y * z;
      dY[12][2] = SH_C3D * (6.f * zz - 3.f * xx - 3.f * yy);
      dY[13][0] = -SH_C3C * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * SH_C3C * x * y;
      dY[13][2] = -8.f * SH_C3C * x * z;
      dY[14][0] = 2.f * SH_C3E * x * z; dY[14][1] = -2.f * SH_C3E * y * z;
      dY[14][2] = SH_C3E * (xx - yy);
      dY[15][0] = -SH_C3A * (3.f * xx - 3.f * yy); dY[15][1] = 6.f * SH_C3A * x * y;
      dY[15][2] = 0.f;
    }
  }
}

// Rotation from a quaternion (w, x, y, z) already normalised; row-major.
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float *R) {
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// ------------------------------------------------------------------------------------------
// Launchers (one per stage), implemented in the .cu files.
struct GaussPtrs {
  const float *means, *scales, *quats, *opacities, *sh;
  int64_t n;
  int32_t sh_degree;
};

int sm_count();
// Per-view parameter table from the caller's cameras; false if any camera is invalid.
bool build_views(const fgs_camera *cams, int n_views, Views *vs);

cudaError_t launch_preprocess_fwd(const GaussPtrs &g, const Views &vs, fgs_record *records,
                                  uint32_t *tiles_touched, cudaStream_t st);
cudaError_t launch_bin_sort(const fgs_record *records, const uint32_t *tiles_touched,
                            int64_t n, const Views &vs, uint64_t *keys, uint32_t *vals,
                            int64_t capacity, uint32_t *tile_ranges, int64_t *n_int,
                            char *ws, const WsLayout &L, uint32_t flags,
                            const CallOpts &opt, cudaStream_t st);
cudaError_t launch_bin_sort_onesweep(const fgs_record *records, const uint32_t *tiles_touched,
                                     int64_t n, const Views &vs, uint64_t *keys,
                                     uint32_t *vals, int64_t capacity, uint32_t *tile_ranges,
                                     int64_t *n_int, char *ws, const WsLayout &L,
                                     const CallOpts &opt, cudaStream_t st);
cudaError_t launch_raster_fwd(const fgs_record *records, const uint32_t *vals,
                              const uint32_t *tile_ranges, const Views &vs, float bg0, float bg1,
                              float bg2, float *images, float *final_T, uint32_t *n_processed,
                              char *ws, const WsLayout &L, const CallOpts &opt,
                              cudaStream_t st);
cudaError_t launch_raster_bwd(const fgs_record *records, const uint32_t *vals,
                              const uint32_t *tile_ranges, const Views &vs, float bg0, float bg1,
                              float bg2, const float *final_T, const uint32_t *n_processed,
                              const float *dL_dimages, int64_t n_records, char *ws,
                              const WsLayout &L, const CallOpts &opt, cudaStream_t st);
cudaError_t launch_preprocess_bwd(const GaussPtrs &g, const Views &vs, const fgs_record *records,
                                  const uint32_t *tiles_touched, const float *g2d,
                                  float *d_means, float *d_scales, float *d_quats,
                                  float *d_opacities, float *d_sh, uint32_t *status,
                                  cudaStream_t st);

}  // namespace fgs
