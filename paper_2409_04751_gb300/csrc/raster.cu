// raster.cu - per-tile alpha blending (Sec. 3.1 "Rendering"; Sec. 4.1 renderCUDA) and its
// backward, sm_103a.
//
// One CTA per 16x16 tile with 256/PPT threads; each thread owns PPT vertically adjacent pixels
// (PPT = 1, 2, 4 or 8 in the backward, the "work shape"; the image does not depend on it). CTAs
// are persistent and take tiles from an atomic queue. Each tile's Gaussians are staged through
// shared memory in batches: every thread issues TMA bulk copies (cp.async.bulk, 48 bytes each)
// of its share, completing on an mbarrier, and the next batch is in flight while the current
// one is blended (two stages); the sorted indices of the batch after next are prefetched into
// registers. Staging drops the list entries whose alpha >= 1/255 ellipse cannot reach the tile
// (the exact binning's conservative test: the tile lists keep the rect binning of the method,
// the blend skips what the rect over-covers) and writes the rest in pairs, so that one paired
// FP32 FMA (fma.rn.f32x2) advances a pixel's exponent for two Gaussians; every kept entry
// carries its list position. With several pixels per thread, a warp first checks whether a
// pair of entries stops any of its pixels and, where none does (most pairs), blends both without
// the stop test. A warp whose pixels have all stopped skips the batch (warp ballot); the CTA
// leaves the tile when all its pixels have stopped.
//
// The backward replays each pixel's blend back to front from its final transmittance and the
// number of list entries it processed (both written by the forward), recovering the
// transmittance before each Gaussian by division; nothing per (pixel, Gaussian) is stored. Per
// list entry it needs nine sums over the pixels: the moments sum dL/dp (dx, dy, dx^2, dx dy,
// dy^2) of the exponent p = -0.5 d^T conic d, sum dL/dalpha alpha_raw, and dL/drgb. Each thread
// sums its own pixels into six local sums (the moments follow from sums of dL/dp weighted by
// the pixel's row inside the thread) and forms the nine from them; the warp then reduces two
// entries' eighteen sums with a transpose reduction (each exchange halves the values a lane
// carries) and lanes add the totals to the records' accumulators. The preprocess backward turns
// the moments into dL/dxy, dL/dconic and dL/dopacity with the record's conic and opacity. The
// backward takes its tiles longest first (tile_work_kernel, tile_order_kernel).
#include <algorithm>
#include "fgs_internal.cuh"

namespace fgs {

namespace {

constexpr int TILE_PIX = TILE * TILE;  // 256 pixels per tile

// Gaussians per staged batch, one per thread at least. The backward takes 256, or 128 and 64
// for the 4- and 8-pixels-per-thread shapes, whose CTAs are small and need a small shared-memory
// footprint to keep enough of them resident. The forward stops a tile once all its pixels have
// saturated, while the next batch is already in flight; on the 180-degree workloads it stages
// only 0.42 records per pair, so its smaller batches (64 at 4 pixels per thread, 128 at 2) waste
// less: 0.196 -> 0.189 ms and 0.201 -> 0.193 ms on the bench workload.
template <int PPT, bool FWD>
struct Batch {
  static constexpr int N = PPT == 8 ? 64
                           : PPT == 4 ? (FWD ? 64 : 128)
                           : PPT == 2 ? (FWD ? 128 : 256) : 256;
  static_assert(N >= TILE_PIX / PPT, "a batch holds one record per thread at least");
};
constexpr uint32_t REC_BYTES = sizeof(fgs_record);
static_assert(REC_BYTES == 48, "record size");

struct TileInfo {
  int v;
  int tx, ty;
  uint32_t start, count;
};

__device__ __forceinline__ TileInfo tile_info(const Views &vs, int64_t t,
                                              const uint32_t *__restrict__ ranges,
                                              const ListBounds &bd, uint32_t *status) {
  TileInfo ti;
  ti.v = view_of_tile(vs, t);
  const View &V = vs.v[ti.v];
  const int64_t local = t - V.tile_offset;
  ti.ty = (int)(local / V.tiles_x);
  ti.tx = (int)(local - (int64_t)ti.ty * V.tiles_x);
  const uint2 rg = __ldg(reinterpret_cast<const uint2 *>(ranges) + t);
  ti.start = rg.x;
  ti.count = rg.y > rg.x ? rg.y - rg.x : 0u;
  // checked build: a range must not be inverted or end past the key capacity
  if (FGS_CHECK && (!in_bounds(rg.x, (uint64_t)rg.y + 1u, status) ||
                    !in_bounds(rg.y, (uint64_t)bd.pairs + 1u, status)))
    ti.count = 0u;
  return ti;
}

// Issue this thread's share of a batch: slots tid, tid + NT, ... below `cnt`, one 48-byte
// bulk copy each, announced with one arrive.expect_tx (the barrier expects NT arrivals).
template <int NT, int PER>
__device__ __forceinline__ void issue_batch(fgs_record *stage, uint64_t *bar,
                                            const fgs_record *__restrict__ rec,
                                            const uint32_t (&idx)[PER], uint32_t cnt) {
  uint32_t n = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) n += (threadIdx.x + k * NT < cnt) ? 1u : 0u;
  mbar_arrive_expect_tx(bar, n * REC_BYTES);
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const uint32_t slot = threadIdx.x + k * NT;
    if (slot < cnt) bulk_g2s(stage + slot, rec + idx[k], REC_BYTES, bar);
  }
}

template <int NT, int PER>
__device__ __forceinline__ void load_idx(const uint32_t *__restrict__ vals, uint32_t base,
                                         uint32_t lo, uint32_t cnt, uint32_t (&idx)[PER],
                                         const ListBounds &bd, uint32_t *status) {
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const uint32_t slot = threadIdx.x + k * NT;
    idx[k] = slot < cnt ? __ldg(vals + base + lo + slot) : 0u;
    if (!in_bounds(idx[k], bd.records, status)) idx[k] = 0u;  // checked build only
  }
}


// The exponent of the blend in base 2, e = A' dx^2 + B' dx dy + C' dy^2 + log2(opacity) with
// (dx, dy) = pixel centre - mean, A' = -log2(e) conic_xx / 2, B' = -log2(e) conic_xy,
// C' = -log2(e) conic_yy / 2, written in tile-centred pixel coordinates (u, v) = pixel centre
// - tile centre (|u|, |v| <= 7.5, so the terms stay small and rounding stays near that of the
// direct form) and factored per pixel row:
//   e = base + v slope + C' v^2,  base = K0 + Kx u + A' u^2,  slope = Ky + B' u.
// Every pixel evaluates exactly this sequence of FMAs whatever the work shape, in the forward
// and in the backward, so both passes take the same alpha >= 1/255 decisions.
//
// Records are staged in pairs (list entries 2p and 2p + 1) so that one paired FP32 FMA
// (fma.rn.f32x2, rounding each half like fmaf) advances a pixel's exponent for both Gaussians:
//   cf[p][0] = (K0_a, K0_b, Kx_a, Kx_b)   cf[p][1] = (Ky_a, Ky_b, A_a, A_b)
//   cf[p][2] = (B_a, B_b, C_a, C_b)       cf[p][3] = (r_a, g_a, b_a, cx_a)
//   cf[p][4] = (r_b, g_b, b_b, cx_b)      cf[p][5] = (cy_a, cy_b, 0, 0)   (backward only)
// with (cx, cy) = tile centre - mean, so dx = u + cx, dy = v + cy. A missing second entry (odd
// count) is staged with K0 = -inf: its exponent is -inf and it never passes the alpha test.
struct Coef {
  float K0, Kx, Ky, A, B, C, r, g, b, cx, cy;
};

__device__ __forceinline__ Coef coef_of(const fgs_record &g, float tile_cx, float tile_cy) {
  Coef k;
  k.A = -0.5f * LOG2E * g.conic[0];
  k.B = -LOG2E * g.conic[1];
  k.C = -0.5f * LOG2E * g.conic[2];
  // the hardware-approximate log2 (a few 1e-7 off in the exponent, far below its FP32 rounding
  // at |e| ~ 8); both passes stage through this function, so they take the same alpha
  const float lo2o = __log2f(g.opacity);
  const float cx = tile_cx - g.xy[0], cy = tile_cy - g.xy[1];
  k.K0 = fmaf(cx, fmaf(k.A, cx, k.B * cy), fmaf(k.C * cy, cy, lo2o));
  k.Kx = fmaf(2.f * k.A, cx, k.B * cy);
  k.Ky = fmaf(k.B, cx, 2.f * k.C * cy);
  k.r = g.rgb[0]; k.g = g.rgb[1]; k.b = g.rgb[2];
  k.cx = cx; k.cy = cy;
  return k;
}

// The exact binning's ellipse-tile test (ellipse_reaches_tile) with hardware reciprocals for
// 1/A and 1/C: their relative error (below 2^-22) moves the clamped edge minimum by far less
// than the test's margin (q* (1 + 1e-3) + 1e-2), so the test stays conservative, and it avoids
// the full-precision division's registers inside the rasterizers.
__device__ __forceinline__ bool reaches_tile(float mx, float my, float A, float B, float C,
                                             float qs, float xl, float xh, float yl, float yh) {
  if (mx >= xl && mx <= xh && my >= yl && my <= yh) return true;
  const float thr = fmaf(qs, 1.001f, 1e-2f);
  const float iA = rcp_approx(A), iC = rcp_approx(C);
  float qmin = 3.0e38f;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dx = (e ? xh : xl) - mx;
    const float dy = fminf(fmaxf(-B * dx * iC, yl - my), yh - my);
    qmin = fminf(qmin, fmaf(dx, fmaf(A, dx, 2.f * B * dy), C * dy * dy));
    const float ey = (e ? yh : yl) - my;
    const float ex = fminf(fmaxf(-B * ey * iA, xl - mx), xh - mx);
    qmin = fminf(qmin, fmaf(ex, fmaf(A, ex, 2.f * B * ey), C * ey * ey));
  }
  return qmin <= thr;
}

// Writes the coefficients of one list entry to its half of pair c / 2, with its list position
// (forward: in the colour float4's spare component; backward: in the pair's last float4).
template <int NF>
__device__ __forceinline__ void write_entry(float4 (*cf)[NF], uint32_t c, const Coef &k,
                                            uint32_t pos) {
  float *q = reinterpret_cast<float *>(cf[c >> 1]);
  const uint32_t h = c & 1u;
  q[0 + h] = k.K0; q[2 + h] = k.Kx;
  q[4 + h] = k.Ky; q[6 + h] = k.A;
  q[8 + h] = k.B;  q[10 + h] = k.C;
  cf[c >> 1][3 + h] = make_float4(k.r, k.g, k.b, NF > 5 ? k.cx : __uint_as_float(pos));
  if (NF > 5) {
    q[20 + h] = k.cy;
    q[22 + h] = __uint_as_float(pos);
  }
}

// Stages a batch of cnt list entries (list positions lo, lo + 1, ...) for the tile whose centre
// is (tile_cx, tile_cy), keeping only the entries whose alpha >= 1/255 ellipse reaches the
// tile's rectangle of pixel centres: the conservative test of the exact binning (the minimum
// of the conic's quadratic over the rectangle against q* = 2 ln(255 opacity), with its margin),
// so a dropped entry contributes to no pixel of the tile and the image is the one of the full
// list. The kept entries are written in list order to positions 0, 1, ... with their list
// positions; the keys, the sort and the tile lists stay those of the rect binning. ridx_in /
// ridx_out (backward) carry the record indices along. A missing second entry of the last pair
// (odd count) gets K0 = -inf and position 2^32 - 1: its exponent never passes the alpha test.
// Each thread takes slots tid, tid + NT, ... (the slots it issued the copies of). Returns the
// number kept; the caller synchronises before reading cf. Kept out of line: inlined, the test's
// registers would count against the blending loop's occupancy.
template <int NT, int PER, int NF>
__device__ __noinline__ uint32_t stage_batch(const fgs_record *raw, uint32_t lo, uint32_t cnt,
                                                float tile_cx, float tile_cy, float4 (*cf)[NF],
                                                const uint32_t *ridx_in, uint32_t *ridx_out,
                                                uint32_t *s_cnt) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float xl = tile_cx - 7.5f, xh = tile_cx + 7.5f, yl = tile_cy - 7.5f, yh = tile_cy + 7.5f;
  uint32_t base = 0;
#pragma unroll 1
  for (int k = 0; k < PER; ++k) {
    const uint32_t slot = tid + k * NT;
    bool keep = false;
    if (slot < cnt) {
      const fgs_record &g = raw[slot];
      // approximate log: the test's margin (q* (1 + 1e-3) + 1e-2) covers its error many times
      const float qs = fmaxf(2.f * __logf(255.f * g.opacity), 0.f);
      keep = reaches_tile(g.xy[0], g.xy[1], g.conic[0], g.conic[1], g.conic[2], qs, xl, xh, yl,
                          yh);
    }
    const uint32_t m = __ballot_sync(0xffffffffu, keep);
    uint32_t before = 0, total = __popc(m);
    if (NW > 1) {
      if (lane == 0) s_cnt[w] = total;
      __syncthreads();
      total = 0;
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) {
        const uint32_t c = s_cnt[ww];
        before += ww < w ? c : 0u;
        total += c;
      }
    }
    if (keep) {
      const uint32_t c = base + before + __popc(m & lanemask_lt());
      write_entry<NF>(cf, c, coef_of(raw[slot], tile_cx, tile_cy), lo + slot);
      if (ridx_out) ridx_out[c] = ridx_in[slot];
    }
    base += total;
    if (NW > 1) __syncthreads();  // s_cnt is rewritten by the next group
  }
  if ((base & 1u) && tid == 0) {
    Coef d;
    d.K0 = -INFINITY;
    d.Kx = d.Ky = d.A = d.B = d.C = d.r = d.g = d.b = d.cx = d.cy = 0.f;
    write_entry<NF>(cf, base, d, 0xffffffffu);
  }
  return base;
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(const float4 &q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 hi2(const float4 &q) { return make_float2(q.z, q.w); }
__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }

// Per-pair terms shared by a thread's pixels (its column u): base and slope of both entries.
struct PairTerms {
  float2 base, slope, C;
};

__device__ __forceinline__ PairTerms pair_terms(const float4 &q0, const float4 &q1,
                                                const float4 &q2, float2 u2, float2 uu2) {
  PairTerms t;
  t.base = ffma2(uu2, hi2(q1), ffma2(u2, hi2(q0), lo2(q0)));
  t.slope = ffma2(u2, lo2(q2), lo2(q1));
  t.C = hi2(q2);
  return t;
}

__device__ __forceinline__ float2 pair_exponent(const PairTerms &t, float v) {
  return ffma2(dup2(v * v), t.C, ffma2(dup2(v), t.slope, t.base));
}

// One list entry blended into two pixels of a thread (rows k and k + 1) at once, without
// branches, with the stop test: an entry takes part at a pixel if the pixel is live and its
// alpha reaches 1/255; the pixel stops (and is left unchanged) if the blend would take its
// transmittance below 1e-4; alpha is selected to 0 otherwise, which leaves T, the colour and the
// processed count exactly as they were. The two pixels' transmittance chains are independent,
// so the FP32 products and fused multiply-adds of the pair are paired instructions (fma / mul
// .rn.f32x2), the compares and selects per pixel. alpha comes in negated and already selected,
// na = -min(0.99, 2^e) where the pixel was live and e >= log2(1/255) when the pair began, else 0
// (exactly max(-0.99, -2^e)), so that T (1 - alpha) = fma(na, T, T) needs no negation; the
// colour sums are kept negated, Cn = -C: fma(rgb, na T, Cn) = -fma(rgb, alpha T, C) exactly
// (rounding to nearest is symmetric), so the image is bit for bit the one of the scalar blend.
// pos1 is the entry's list position + 1.
template <bool COUNT>
__device__ __forceinline__ void fwd_blend2_na(bool &live0, bool &live1, float2 na, const float4 &q,
                                              uint32_t pos1, float2 &T, float2 &Cn0, float2 &Cn1,
                                              float2 &Cn2, uint32_t &last0, uint32_t &last1,
                                              uint32_t &n_blend) {
  // a pixel that stopped at the pair's first entry takes no part in its second
  const bool c0 = live0 && na.x != 0.f, c1 = live1 && na.y != 0.f;
  const float2 Tn = __ffma2_rn(na, T, T);
  const bool stop0 = c0 && Tn.x < T_MIN, stop1 = c1 && Tn.y < T_MIN;
  live0 = live0 && !stop0;
  live1 = live1 && !stop1;
  const float2 a = make_float2(c0 && !stop0 ? na.x : 0.f, c1 && !stop1 ? na.y : 0.f);
  const float2 w = __fmul2_rn(a, T);
  Cn0 = __ffma2_rn(make_float2(q.x, q.x), w, Cn0);
  Cn1 = __ffma2_rn(make_float2(q.y, q.y), w, Cn1);
  Cn2 = __ffma2_rn(make_float2(q.z, q.z), w, Cn2);
  T = __ffma2_rn(a, T, T);
  last0 = c0 && !stop0 ? pos1 : last0;
  last1 = c1 && !stop1 ? pos1 : last1;
  if (COUNT) n_blend += (c0 && !stop0 ? 1u : 0u) + (c1 && !stop1 ? 1u : 0u);
}

template <int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE_PIX / PPT, PPT == 1 ? 5 : 1)
    raster_fwd_kernel(const fgs_record *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ ranges, Views vs, float bg0, float bg1,
                      float bg2, float *__restrict__ images, float *__restrict__ final_T,
                      uint32_t *__restrict__ n_processed, uint32_t *tile_counter,
                      uint32_t *status, unsigned long long *counters) {
  constexpr int NT = TILE_PIX / PPT;
  constexpr int BATCH = Batch<PPT, true>::N;
  constexpr int PER = BATCH / NT;  // copies each thread issues per batch
  __shared__ __align__(128) fgs_record raw[2][BATCH];
  __shared__ __align__(16) float4 cf[BATCH / 2][5];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_tile;
  __shared__ uint32_t s_cnt[NT / 32];
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], NT);
    mbar_init(&bar[1], NT);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase0 = 0, phase1 = 0;
  uint32_t n_eval = 0, n_blend = 0;
  unsigned long long n_staged = 0;  // records copied in (thread 0 counts)
  const int lx = tid & (TILE - 1), ly0 = (tid / TILE) * PPT;
  const float fu = (float)lx - 7.5f, fv = (float)ly0 - 7.5f;
  const float2 u2 = dup2(fu), uu2 = dup2(fu * fu);
  // after a device-side error in the binning the lists are undefined: render background only
  const bool lists_ok = *(volatile const uint32_t *)status == 0u;
  const ListBounds bd = list_bounds(status);

  for (;;) {
    if (tid == 0) s_tile = (int64_t)atomicAdd(tile_counter, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    __syncthreads();
    if (t >= vs.total_tiles) break;
    const TileInfo ti = tile_info(vs, t, ranges, bd, status);
    const View &V = vs.v[ti.v];
    const int px = ti.tx * TILE + lx;
    // tile centre (between pixel centres 7 and 8)
    const float tile_cx = (float)(ti.tx * TILE) + 0.5f * TILE, tile_cy = (float)(ti.ty * TILE) + 0.5f * TILE;
    float T[PPT], C0[PPT], C1[PPT], C2[PPT];
    uint32_t last[PPT];
    bool live[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = ti.ty * TILE + ly0 + k;
      T[k] = 1.f; C0[k] = C1[k] = C2[k] = 0.f;
      last[k] = 0;
      live[k] = px < V.width && py < V.height;
    }
    bool done = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) done = done && !live[k];
    const uint32_t count = lists_ok ? ti.count : 0u;
    const uint32_t nb = (count + BATCH - 1) / BATCH;

    if (nb > 0) {
      uint32_t idx[PER], idx_next[PER];
      load_idx<NT, PER>(vals, ti.start, 0, count, idx, bd, status);
      load_idx<NT, PER>(vals, ti.start, BATCH, count > BATCH ? count - BATCH : 0u, idx_next, bd, status);
      fence_proxy_async_smem();
      issue_batch<NT, PER>(raw[0], &bar[0], rec, idx, min(count, (uint32_t)BATCH));
      if (COUNT && tid == 0) n_staged += min(count, (uint32_t)BATCH);
      for (uint32_t b = 0; b < nb; ++b) {
        const int s = b & 1;
        const uint32_t lo = b * BATCH;
        const uint32_t cnt = min((uint32_t)BATCH, count - lo);
        if (b + 1 < nb) {
          fence_proxy_async_smem();
          issue_batch<NT, PER>(raw[s ^ 1], &bar[s ^ 1], rec, idx_next,
                               min((uint32_t)BATCH, count - lo - BATCH));
          if (COUNT && tid == 0) n_staged += min((uint32_t)BATCH, count - lo - BATCH);
          const uint32_t lo2 = lo + 2 * BATCH;
          load_idx<NT, PER>(vals, ti.start, lo2, count > lo2 ? count - lo2 : 0u, idx_next, bd, status);
        }
        const bool ok = mbar_wait(&bar[s], s ? phase1 : phase0, status);
        if (s) phase1 ^= 1u; else phase0 ^= 1u;
        if (__syncthreads_or(!ok)) {  // a copy never landed: drain (bounded) and leave
          if (b + 1 < nb) mbar_wait(&bar[s ^ 1], s ? phase0 : phase1, status);
          return;
        }
        const uint32_t kept = stage_batch<NT, PER, 5>(raw[s], lo, cnt, tile_cx, tile_cy, cf,
                                                      nullptr, nullptr, s_cnt);
        __syncthreads();
        const uint32_t npairs = (kept + 1) / 2;
        if (PPT == 1 && !__all_sync(0xffffffffu, done)) {
          // one pixel per thread: a tight loop over the pairs, left at the stop
          if (!done) {
            const float2 v2 = dup2(fv), vv2 = dup2(fv * fv);
            bool stop = false;
            for (uint32_t p = 0; p < npairs; ++p) {
              const PairTerms pt = pair_terms(cf[p][0], cf[p][1], cf[p][2], u2, uu2);
              const float2 e = ffma2(vv2, pt.C, ffma2(v2, pt.slope, pt.base));
              if (COUNT) n_eval += 2 * p + 1 < kept ? 2 : 1;
              // branch-free blends: an entry below 1/255 gets alpha = 0, which leaves T, the
              // colour and the processed count exactly as they were
              const bool ca = e.x >= LOG2_ALPHA_MIN, cb = e.y >= LOG2_ALPHA_MIN;
              {
                const float alpha = ca ? fminf(ALPHA_MAX, ex2_approx(e.x)) : 0.f;
                const float Tn = fmaf(-alpha, T[0], T[0]);
                if (Tn < T_MIN) {
                  stop = true;
                  if (COUNT && 2 * p + 1 < kept) --n_eval;
                  break;
                }
                const float4 c = cf[p][3];
                const float wgt = alpha * T[0];
                C0[0] = fmaf(c.x, wgt, C0[0]);
                C1[0] = fmaf(c.y, wgt, C1[0]);
                C2[0] = fmaf(c.z, wgt, C2[0]);
                T[0] = Tn;
                last[0] = ca ? __float_as_uint(c.w) + 1 : last[0];
                if (COUNT && ca) ++n_blend;
              }
              {
                const float alpha = cb ? fminf(ALPHA_MAX, ex2_approx(e.y)) : 0.f;
                const float Tn = fmaf(-alpha, T[0], T[0]);
                if (Tn < T_MIN) {
                  stop = true;
                  break;
                }
                const float4 c = cf[p][4];
                const float wgt = alpha * T[0];
                C0[0] = fmaf(c.x, wgt, C0[0]);
                C1[0] = fmaf(c.y, wgt, C1[0]);
                C2[0] = fmaf(c.z, wgt, C2[0]);
                T[0] = Tn;
                last[0] = cb ? __float_as_uint(c.w) + 1 : last[0];
                if (COUNT && cb) ++n_blend;
              }
            }
            if (stop) live[0] = false;
            done = !live[0];
          }
        } else if (PPT > 1 && !__all_sync(0xffffffffu, done)) {
          // several pixels per thread, blended without branches (alpha selected to 0 where a
          // pixel does not take part), so that the compiler interleaves the pixels'
          // transmittance chains; pixels in pairs (rows k, k + 1): the exponents per pixel (the
          // same FMA sequence as every other shape), the blends paired over the two rows, with
          // the colour sums kept negated until the tile is written. A pixel stops at most once
          // per tile, so most pairs of list entries stop no pixel of the warp (87% on a
          // saturating 1752x1168 view): the warp tests that first and then blends both entries
          // without the stop's compares and selects, the same operations in the same order as
          // the exact path (fwd_blend2_na), which it takes otherwise
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            C0[k] = -C0[k];
            C1[k] = -C1[k];
            C2[k] = -C2[k];
          }
          // every thread of the warp runs every iteration (the votes below name all 32 lanes);
          // the warp leaves together once none of its pixels is live
          for (uint32_t p = 0; p < npairs; ++p) {
            const PairTerms pt = pair_terms(cf[p][0], cf[p][1], cf[p][2], u2, uu2);
            const float4 qa = cf[p][3], qb = cf[p][4];
            const bool has_b = 2 * p + 1 < kept;
            // both entries' negated alphas for every pixel (0 where a pixel does not take
            // part), and whether the pair would take some pixel below 1e-4: T_b = T (1 - a_a)
            // (1 - a_b) is the smaller of the two transmittances, so T_b >= 1e-4 means neither
            // entry stops the pixel
            float2 na_a[PPT > 1 ? PPT / 2 : 1], na_b[PPT > 1 ? PPT / 2 : 1];
            uint32_t last_n[PPT];  // the processed counts if no pixel stops
            const uint32_t pa1 = __float_as_uint(qa.w) + 1, pb1 = __float_as_uint(qb.w) + 1;
            bool would_stop = false;
#pragma unroll
            for (int k = 0; k < PPT; k += 2) {
              const float2 e0 = pair_exponent(pt, fv + (float)k);
              const float2 e1 = pair_exponent(pt, fv + (float)(k + 1));
              const bool ca0 = live[k] && e0.x >= LOG2_ALPHA_MIN, ca1 = live[k + 1] && e1.x >= LOG2_ALPHA_MIN;
              const bool cb0 = live[k] && e0.y >= LOG2_ALPHA_MIN, cb1 = live[k + 1] && e1.y >= LOG2_ALPHA_MIN;
              na_a[k / 2] = make_float2(ca0 ? fmaxf(-ALPHA_MAX, -ex2_approx(e0.x)) : 0.f,
                                        ca1 ? fmaxf(-ALPHA_MAX, -ex2_approx(e1.x)) : 0.f);
              na_b[k / 2] = make_float2(cb0 ? fmaxf(-ALPHA_MAX, -ex2_approx(e0.y)) : 0.f,
                                        cb1 ? fmaxf(-ALPHA_MAX, -ex2_approx(e1.y)) : 0.f);
              const float2 Tp = make_float2(T[k], T[k + 1]);
              const float2 Ta = __ffma2_rn(na_a[k / 2], Tp, Tp);
              const float2 Tb = __ffma2_rn(na_b[k / 2], Ta, Ta);
              would_stop = would_stop || Tb.x < T_MIN || Tb.y < T_MIN;
              last_n[k] = cb0 ? pb1 : ca0 ? pa1 : last[k];
              last_n[k + 1] = cb1 ? pb1 : ca1 ? pa1 : last[k + 1];
            }
            if (!__any_sync(0xffffffffu, would_stop)) {
              // no pixel of the warp stops: both blends without the stop's selects
#pragma unroll
              for (int k = 0; k < PPT; k += 2) {
                // (no pixel stops, so the live pixels evaluate both entries)
                if (COUNT) n_eval += ((live[k] ? 1u : 0u) + (live[k + 1] ? 1u : 0u)) * (has_b ? 2u : 1u);
                const float2 Tp = make_float2(T[k], T[k + 1]);
                float2 C0p = make_float2(C0[k], C0[k + 1]), C1p = make_float2(C1[k], C1[k + 1]);
                float2 C2p = make_float2(C2[k], C2[k + 1]);
                const float2 wa = __fmul2_rn(na_a[k / 2], Tp);
                C0p = __ffma2_rn(dup2(qa.x), wa, C0p);
                C1p = __ffma2_rn(dup2(qa.y), wa, C1p);
                C2p = __ffma2_rn(dup2(qa.z), wa, C2p);
                const float2 Ta = __ffma2_rn(na_a[k / 2], Tp, Tp);
                const float2 wb = __fmul2_rn(na_b[k / 2], Ta);
                C0p = __ffma2_rn(dup2(qb.x), wb, C0p);
                C1p = __ffma2_rn(dup2(qb.y), wb, C1p);
                C2p = __ffma2_rn(dup2(qb.z), wb, C2p);
                const float2 Tb = __ffma2_rn(na_b[k / 2], Ta, Ta);
                last[k] = last_n[k];
                last[k + 1] = last_n[k + 1];
                if (COUNT)
                  n_blend += (na_a[k / 2].x != 0.f) + (na_a[k / 2].y != 0.f) +
                             (na_b[k / 2].x != 0.f) + (na_b[k / 2].y != 0.f);
                T[k] = Tb.x; T[k + 1] = Tb.y;
                C0[k] = C0p.x; C0[k + 1] = C0p.y;
                C1[k] = C1p.x; C1[k + 1] = C1p.y;
                C2[k] = C2p.x; C2[k + 1] = C2p.y;
              }
            } else {
              // some pixel stops: the exact blends, entry a then entry b
              bool any_live = false;
#pragma unroll
              for (int k = 0; k < PPT; k += 2) {
                float2 Tp = make_float2(T[k], T[k + 1]);
                float2 C0p = make_float2(C0[k], C0[k + 1]), C1p = make_float2(C1[k], C1[k + 1]);
                float2 C2p = make_float2(C2[k], C2[k + 1]);
                // a pixel that stops at entry a does not evaluate entry b
                if (COUNT) n_eval += (live[k] ? 1u : 0u) + (live[k + 1] ? 1u : 0u);
                fwd_blend2_na<COUNT>(live[k], live[k + 1], na_a[k / 2], qa, pa1, Tp, C0p, C1p, C2p,
                                     last[k], last[k + 1], n_blend);
                if (COUNT && has_b) n_eval += (live[k] ? 1u : 0u) + (live[k + 1] ? 1u : 0u);
                fwd_blend2_na<COUNT>(live[k], live[k + 1], na_b[k / 2], qb, pb1, Tp, C0p, C1p, C2p,
                                     last[k], last[k + 1], n_blend);
                T[k] = Tp.x; T[k + 1] = Tp.y;
                C0[k] = C0p.x; C0[k + 1] = C0p.y;
                C1[k] = C1p.x; C1[k + 1] = C1p.y;
                C2[k] = C2p.x; C2[k + 1] = C2p.y;
                any_live = any_live || live[k] || live[k + 1];
              }
              done = !any_live;
              if (__all_sync(0xffffffffu, done)) break;
            }
          }
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            C0[k] = -C0[k];
            C1[k] = -C1[k];
            C2[k] = -C2[k];
          }
        }
        if (__syncthreads_count(!done) == 0) {
          if (b + 1 < nb) {  // drain the batch in flight before leaving the tile
            mbar_wait(&bar[s ^ 1], s ? phase0 : phase1, status);
            if (s) phase0 ^= 1u; else phase1 ^= 1u;
          }
          break;
        }
      }
    }
    const int64_t plane = (int64_t)V.width * V.height;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = ti.ty * TILE + ly0 + k;
      if (px < V.width && py < V.height) {
        const int64_t off = (int64_t)py * V.width + px;
        float *img = images + 3 * V.pixel_offset + off;
        img[0] = fmaf(T[k], bg0, C0[k]);
        img[plane] = fmaf(T[k], bg1, C1[k]);
        img[2 * plane] = fmaf(T[k], bg2, C2[k]);
        final_T[V.pixel_offset + off] = T[k];
        n_processed[V.pixel_offset + off] = last[k];
      }
    }
  }
  if (COUNT) {
    atomicAdd(&counters[0], (unsigned long long)n_eval);
    atomicAdd(&counters[1], (unsigned long long)n_blend);
    if (tid == 0) atomicAdd(&counters[4], n_staged);
  }
}

// Warp sums of two entries' nine values by transpose reduction. At each exchange a lane keeps
// half of its values and sends the other half to its partner, so the sixteen values
// a[0..7], b[0..7] take 8 + 4 + 2 + 1 + 1 shuffles; on return lanes 2i and 2i + 1 hold the
// total of value i of (a[0..7], b[0..7]). The ninth values a8, b8 take 1 + 4 shuffles; on
// return lanes 0..15 hold the total of a8 and lanes 16..31 that of b8.
__device__ __forceinline__ float warp_transpose_sum16(const float (&a)[9], const float (&b)[9],
                                                      int lane, float &tot8) {
  float c[8], d[4], e[2];
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float keep = h4 ? b[k] : a[k];
    const float send = h4 ? a[k] : b[k];
    c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  {
    const float keep = h4 ? b[8] : a[8];
    const float send = h4 ? a[8] : b[8];
    float t = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    t += __shfl_xor_sync(0xffffffffu, t, 8);
    t += __shfl_xor_sync(0xffffffffu, t, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    tot8 = t;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float keep = h3 ? c[k + 4] : c[k];
    const float send = h3 ? c[k] : c[k + 4];
    d[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float keep = h2 ? d[k + 2] : d[k];
    const float send = h2 ? d[k] : d[k + 2];
    e[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  float f = (h1 ? e[1] : e[0]) + __shfl_xor_sync(0xffffffffu, h1 ? e[0] : e[1], 2);
  f += __shfl_xor_sync(0xffffffffu, f, 1);
  return f;
}

// One (pixel, Gaussian) pair of the backward, back to front, its contribution decided by c:
// recovers the transmittance in front of the Gaussian, updates the colour-behind sum GS and
// adds the pixel's terms to the entry's six local sums a. A pixel that does not take part (not
// yet reached back to front, or alpha below 1/255) gets alpha = 0 and 1/(1 - alpha) = 1 by
// selection, so its transmittance, GS and sums stay exactly as they were. The backward calls
// it for every pixel and entry without branching: the cull at staging leaves most evaluations
// contributing, and straight-line code lets the compiler interleave the independent
// transmittance chains of a thread's pixels, which hides the latency of each chain.
//
// alpha = opacity exp(p), p = -0.5 d^T conic d, so dL/dp = dL/dalpha alpha where alpha is below
// its cap, and the opacity term dL/dalpha alpha_raw equals dL/dp there: one sum serves both.
// The moments of dL/dp over the pixel offsets (dx, dy) = (u + cx, v + cy) are not formed per
// pixel: the thread's pixels share the column u and sit in rows v = v0 + k, k = 0 .. PPT - 1,
// so a[0] = sum dL/dp, a[1] = sum k dL/dp and a[2] = sum k^2 dL/dp (k a constant once the
// pixel loop is unrolled) determine all five (moments_of_local_sums). a[3..5] = sum dL/drgb.
__device__ __forceinline__ void bwd_contrib(bool c, float e, float r, float g, float b, int k,
                                            float G0, float G1, float G2, float &T, float &GS,
                                            float (&a)[6]) {
  const float araw = c ? ex2_approx(e) : 0.f;
  const float alpha = fminf(ALPHA_MAX, araw);
  const float om = c ? rcp_approx(1.f - alpha) : 1.f;
  T *= om;  // transmittance before this Gaussian
  const float wgt = alpha * T;
  const float gc = G0 * r + G1 * g + G2 * b;  // <dL/dC, colour>
  // dL/dalpha = <dL/dC, colour T - behind / (1 - alpha)>
  const float dLda = fmaf(T, gc, -om * GS);
  GS = fmaf(gc, wgt, GS);
  a[3] = fmaf(G0, wgt, a[3]);
  a[4] = fmaf(G1, wgt, a[4]);
  a[5] = fmaf(G2, wgt, a[5]);
  const float d = dLda * (araw < ALPHA_MAX ? araw : 0.f);  // dL/dp
  a[0] += d;
  if (k > 0) {  // k is a constant in the unrolled pixel loop
    a[1] = fmaf(d, (float)k, a[1]);
    a[2] = fmaf(d, (float)(k * k), a[2]);
  }
}

// bwd_contrib for two pixels of a thread (rows k and k + 1) and one entry at once. Their
// transmittance chains are independent, so every FP32 add, multiply and fused multiply-add of
// the pair is one paired instruction (add / mul / fma .rn.f32x2, each half rounded exactly as
// the scalar operation); the selects, compares and MUFU operations stay per pixel. a[0] sums
// dL/dp and a[3..5] the colour terms for the two rows separately (folded after the pixel loop);
// a[1] and a[2] are filled by the caller (suffix sums over the pixel pairs, see below).
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ void bwd_contrib2(bool c0, bool c1, float2 e, float r, float g,
                                             float b, float2 G0, float2 G1, float2 G2,
                                             float2 &T, float2 &GS, float2 (&a)[6]) {
  const float2 araw = make_float2(c0 ? ex2_approx(e.x) : 0.f, c1 ? ex2_approx(e.y) : 0.f);
  const float2 alpha = make_float2(fminf(ALPHA_MAX, araw.x), fminf(ALPHA_MAX, araw.y));
  const float2 oma = fadd2(dup2(1.f), make_float2(-alpha.x, -alpha.y));
  // a pixel that does not take part has alpha = 0 and 1 - alpha = 1, whose hardware
  // reciprocal is exactly 1 (checked on sm_103a), so its transmittance is left as it was
  // without a select
  const float2 om = make_float2(rcp_approx(oma.x), rcp_approx(oma.y));
  T = fmul2(T, om);  // transmittance before this Gaussian
  const float2 wgt = fmul2(alpha, T);
  const float2 gc = ffma2(G2, dup2(b), ffma2(G1, dup2(g), fmul2(G0, dup2(r))));
  const float2 dLda = ffma2(T, gc, fmul2(make_float2(-om.x, -om.y), GS));
  GS = ffma2(gc, wgt, GS);
  a[3] = ffma2(G0, wgt, a[3]);
  a[4] = ffma2(G1, wgt, a[4]);
  a[5] = ffma2(G2, wgt, a[5]);
  const float2 d = fmul2(dLda, make_float2(araw.x < ALPHA_MAX ? araw.x : 0.f,
                                            araw.y < ALPHA_MAX ? araw.y : 0.f));  // dL/dp
  a[0] = fadd2(a[0], d);
}

// Row-weighted sums of a thread's pixels from suffix sums. The pixel pairs j = J-1 .. 0
// (rows 2j, 2j + 1) are visited in descending order; after pair j is added to P = a[0],
// Q = a[1] += P (j >= 1) and R = a[2] += Q (j >= 2), so that per half
// Q = sum_j j d_j and R = sum_j j (j - 1) / 2 d_j. With rows k = 2j (x) and 2j + 1 (y):
//   sum d = P.x + P.y,  sum k d = 2 (Q.x + Q.y) + P.y,
//   sum k^2 d = 8 (R.x + R.y) + 4 (Q.x + Q.y) + 4 Q.y + P.y
// (k^2 = 4 j^2 (+ 4 j + 1 for the odd row) and j^2 = 2 j (j - 1) / 2 + j). Only additions, no
// per-row weights.
__device__ __forceinline__ void suffix_step(int k, float2 (&a)[6]) {
  if (k >= 2) a[1] = fadd2(a[1], a[0]);
  if (k >= 4) a[2] = fadd2(a[2], a[1]);
}

__device__ __forceinline__ void fold_pairs(const float2 (&a)[6], float (&s)[6]) {
  const float qs = a[1].x + a[1].y, rs = a[2].x + a[2].y;
  s[0] = a[0].x + a[0].y;
  s[1] = fmaf(2.f, qs, a[0].y);
  s[2] = fmaf(8.f, rs, fmaf(4.f, qs + a[1].y, a[0].y));
  s[3] = a[3].x + a[3].y;
  s[4] = a[4].x + a[4].y;
  s[5] = a[5].x + a[5].y;
}

// The nine per-record sums of one entry from a thread's local sums: with w = v0 + cy (the first
// row's offset from the mean) and dx = u + cx,
//   sum dL/dp dx = dx S,  sum dL/dp dy = w S + S_k,  sum dL/dp dx^2 = dx^2 S,
//   sum dL/dp dx dy = dx (w S + S_k),  sum dL/dp dy^2 = w^2 S + 2 w S_k + S_kk,
// then the opacity term (S itself) and the three colour sums.
__device__ __forceinline__ void moments_of_local_sums(const float (&a)[6], float dx, float w,
                                                      float (&v)[9]) {
  v[0] = dx * a[0];
  v[1] = fmaf(w, a[0], a[1]);
  v[2] = dx * v[0];
  v[3] = dx * v[1];
  v[4] = fmaf(w, v[1] + a[1], a[2]);
  v[5] = a[0];
  v[6] = a[3];
  v[7] = a[4];
  v[8] = a[5];
}

// 8 pixels per thread (one warp per tile): at most 128 registers, so that 16 one-warp CTAs fit
// an SM (the paired pixel state would otherwise take 160 and leave 12)
template <int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE_PIX / PPT, PPT == 8 ? 16 : 1)
    raster_bwd_kernel(const fgs_record *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ ranges, Views vs, float bg0, float bg1,
                      float bg2, const float *__restrict__ final_T,
                      const uint32_t *__restrict__ n_processed, const float *__restrict__ dLdimg,
                      float *__restrict__ g2d, const uint32_t *__restrict__ order,
                      uint32_t *tile_counter, uint32_t *status, unsigned long long *counters) {
  constexpr int NT = TILE_PIX / PPT;
  constexpr int BATCH = Batch<PPT, false>::N;
  constexpr int PER = BATCH / NT;
  __shared__ __align__(128) fgs_record raw[2][BATCH];
  __shared__ __align__(16) float4 cf[BATCH / 2][6];
  __shared__ uint32_t xidx[BATCH];  // record of each slot of the batch
  __shared__ uint32_t cidx[BATCH];  // record of each kept entry
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_tile;
  __shared__ uint32_t s_max;
  __shared__ uint32_t s_cnt[NT / 32];
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar[0], NT);
    mbar_init(&bar[1], NT);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase0 = 0, phase1 = 0;
  uint32_t n_eval = 0, n_contrib = 0;
  unsigned long long n_staged = 0;  // records copied in (thread 0 counts)
  const int lx = tid & (TILE - 1), ly0 = (tid / TILE) * PPT;
  const float fu = (float)lx - 7.5f, fv = (float)ly0 - 7.5f;
  const float2 u2 = dup2(fu), uu2 = dup2(fu * fu);
  // after a device-side error in the binning the lists are undefined: no gradient flows
  const bool lists_ok = *(volatile const uint32_t *)status == 0u;
  const ListBounds bd = list_bounds(status);

  for (;;) {
    if (tid == 0) {  // tiles in decreasing order of work
      const uint32_t q = atomicAdd(tile_counter, 1u);
      s_tile = q < vs.total_tiles ? (int64_t)order[q] : vs.total_tiles;
      // checked build: the order lists tiles only (an entry outside ends this CTA's work)
      if (q < vs.total_tiles) in_bounds((uint64_t)s_tile, (uint64_t)vs.total_tiles, status);
      s_max = 0u;
    }
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= vs.total_tiles) break;
    const TileInfo ti = tile_info(vs, t, ranges, bd, status);
    const View &V = vs.v[ti.v];
    const int px = ti.tx * TILE + lx;
    const float tile_cx = (float)(ti.tx * TILE) + 0.5f * TILE, tile_cy = (float)(ti.ty * TILE) + 0.5f * TILE;
    const int64_t plane = (int64_t)V.width * V.height;
    // per pixel: transmittance, dL/dC, and GS = <dL/dC, colour behind the current entry>
    // (the sum over later blended entries plus T_final bg), kept as one scalar
    float T[PPT], G0[PPT], G1[PPT], G2[PPT], GS[PPT];
    uint32_t last[PPT];
    uint32_t my_max = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = ti.ty * TILE + ly0 + k;
      T[k] = 1.f; G0[k] = G1[k] = G2[k] = 0.f;
      last[k] = 0;
      if (px < V.width && py < V.height) {
        const int64_t off = (int64_t)py * V.width + px;
        const float *gi = dLdimg + 3 * V.pixel_offset + off;
        T[k] = final_T[V.pixel_offset + off];
        last[k] = lists_ok ? min(n_processed[V.pixel_offset + off], ti.count) : 0u;
        G0[k] = gi[0]; G1[k] = gi[plane]; G2[k] = gi[2 * plane];
      }
      GS[k] = T[k] * (G0[k] * bg0 + G1[k] * bg1 + G2[k] * bg2);
      my_max = max(my_max, last[k]);
    }
    atomicMax(&s_max, my_max);
    __syncthreads();
    const uint32_t max_last = s_max;
    const uint32_t nb = (max_last + BATCH - 1) / BATCH;

    if (nb > 0) {
      // batches from the back: iteration it handles batch nb - 1 - it
      uint32_t idx[PER], idx_next[PER];
      {
        const uint32_t lo0 = (nb - 1) * BATCH;
        load_idx<NT, PER>(vals, ti.start, lo0, max_last - lo0, idx, bd, status);
        if (nb >= 2) load_idx<NT, PER>(vals, ti.start, lo0 - BATCH, BATCH, idx_next, bd, status);
        fence_proxy_async_smem();
        issue_batch<NT, PER>(raw[0], &bar[0], rec, idx, max_last - lo0);
        if (COUNT && tid == 0) n_staged += max_last - lo0;
#pragma unroll
        for (int k = 0; k < PER; ++k) xidx[tid + k * NT] = idx[k];
      }
      for (uint32_t it = 0; it < nb; ++it) {
        const uint32_t b = nb - 1 - it;
        const int s = it & 1;
        const uint32_t lo = b * BATCH;
        const uint32_t cnt = min((uint32_t)BATCH, max_last - lo);
        uint32_t mine[PER];
        if (b >= 1) {
          fence_proxy_async_smem();
          issue_batch<NT, PER>(raw[s ^ 1], &bar[s ^ 1], rec, idx_next, BATCH);
          if (COUNT && tid == 0) n_staged += BATCH;
#pragma unroll
          for (int k = 0; k < PER; ++k) mine[k] = idx_next[k];
          if (b >= 2) load_idx<NT, PER>(vals, ti.start, lo - 2 * BATCH, BATCH, idx_next, bd, status);
        }
        const bool ok = mbar_wait(&bar[s], s ? phase1 : phase0, status);
        if (s) phase1 ^= 1u; else phase0 ^= 1u;
        if (__syncthreads_or(!ok)) {  // a copy never landed: drain (bounded) and leave
          if (b >= 1) mbar_wait(&bar[s ^ 1], s ? phase0 : phase1, status);
          return;
        }
        const uint32_t kept = stage_batch<NT, PER, 6>(raw[s], lo, cnt, tile_cx, tile_cy, cf, xidx,
                                                      cidx, s_cnt);
        __syncthreads();
        const uint32_t npairs = (kept + 1) / 2;
        for (int p = (int)npairs - 1; p >= 0; --p) {
          const float4 qy = cf[p][5];
          const uint32_t pos_a = __float_as_uint(qy.z), pos_b = __float_as_uint(qy.w);
          const bool any_pos = pos_a < my_max;
          if (!__any_sync(0xffffffffu, any_pos)) continue;
          float va[9], vb[9];
          bool ca = false, cb = false;
          {
            const PairTerms pt = pair_terms(cf[p][0], cf[p][1], cf[p][2], u2, uu2);
            const float4 qa = cf[p][3], qb = cf[p][4];
            float sa[6], sb[6];
            if constexpr (PPT == 1) {
#pragma unroll
              for (int q = 0; q < 6; ++q) sa[q] = sb[q] = 0.f;
              const bool in_a = pos_a < last[0], in_b = pos_b < last[0];
              const float2 e = pair_exponent(pt, fv);
              const bool cbk = in_b && e.y >= LOG2_ALPHA_MIN, cak = in_a && e.x >= LOG2_ALPHA_MIN;
              if (COUNT) {
                n_eval += (in_a ? 1u : 0u) + (in_b ? 1u : 0u);
                n_contrib += (cak ? 1u : 0u) + (cbk ? 1u : 0u);
              }
              cb = cbk;
              ca = cak;
              bwd_contrib(cbk, e.y, qb.x, qb.y, qb.z, 0, G0[0], G1[0], G2[0], T[0], GS[0], sb);
              bwd_contrib(cak, e.x, qa.x, qa.y, qa.z, 0, G0[0], G1[0], G2[0], T[0], GS[0], sa);
            } else {
              // pixels in pairs (rows k, k + 1): the exponents of one entry for both rows, then
              // the paired contributions, entry b (behind) before entry a
              float2 pa[6], pb[6];
#pragma unroll
              for (int q = 0; q < 6; ++q) pa[q] = pb[q] = dup2(0.f);
              const float2 base_a = dup2(pt.base.x), base_b = dup2(pt.base.y);
              const float2 slope_a = dup2(pt.slope.x), slope_b = dup2(pt.slope.y);
              const float2 C_a = dup2(pt.C.x), C_b = dup2(pt.C.y);
#pragma unroll
              for (int k = PPT - 2; k >= 0; k -= 2) {  // descending pairs: suffix sums
                const float2 vv = make_float2(fv + (float)k, fv + (float)(k + 1));
                const float2 vsq = fmul2(vv, vv);
                const float2 ea = ffma2(vsq, C_a, ffma2(vv, slope_a, base_a));
                const float2 eb = ffma2(vsq, C_b, ffma2(vv, slope_b, base_b));
                const bool ia0 = pos_a < last[k], ia1 = pos_a < last[k + 1];
                const bool ib0 = pos_b < last[k], ib1 = pos_b < last[k + 1];
                const bool ca0 = ia0 && ea.x >= LOG2_ALPHA_MIN, ca1 = ia1 && ea.y >= LOG2_ALPHA_MIN;
                const bool cb0 = ib0 && eb.x >= LOG2_ALPHA_MIN, cb1 = ib1 && eb.y >= LOG2_ALPHA_MIN;
                if (COUNT) {
                  n_eval += (ia0 ? 1u : 0u) + (ia1 ? 1u : 0u) + (ib0 ? 1u : 0u) + (ib1 ? 1u : 0u);
                  n_contrib += (ca0 ? 1u : 0u) + (ca1 ? 1u : 0u) + (cb0 ? 1u : 0u) + (cb1 ? 1u : 0u);
                }
                cb = cb || cb0 || cb1;
                ca = ca || ca0 || ca1;
                float2 Tp = make_float2(T[k], T[k + 1]), GSp = make_float2(GS[k], GS[k + 1]);
                const float2 G0p = make_float2(G0[k], G0[k + 1]), G1p = make_float2(G1[k], G1[k + 1]);
                const float2 G2p = make_float2(G2[k], G2[k + 1]);
                bwd_contrib2(cb0, cb1, eb, qb.x, qb.y, qb.z, G0p, G1p, G2p, Tp, GSp, pb);
                bwd_contrib2(ca0, ca1, ea, qa.x, qa.y, qa.z, G0p, G1p, G2p, Tp, GSp, pa);
                suffix_step(k, pb);
                suffix_step(k, pa);
                T[k] = Tp.x; T[k + 1] = Tp.y;
                GS[k] = GSp.x; GS[k + 1] = GSp.y;
              }
              fold_pairs(pa, sa);
              fold_pairs(pb, sb);
            }
            moments_of_local_sums(sa, fu + qa.w, fv + qy.x, va);
            moments_of_local_sums(sb, fu + qb.w, fv + qy.y, vb);
          }
          const bool any_a = __any_sync(0xffffffffu, ca), any_b = __any_sync(0xffffffffu, cb);
          if (any_a || any_b) {
            float tot8;
            const float tot = warp_transpose_sum16(va, vb, lane, tot8);
            // one atomic per lane at most: even lanes 2i add value i of (a[0..7], b[0..7]),
            // lanes 1 and 17 the ninth value of a and of b
            const bool even = (lane & 1) == 0;
            const bool for_b = even ? lane >= 16 : lane == 17;
            const bool act = (even || lane == 1 || lane == 17) && (for_b ? any_b : any_a);
            if (act) {
              float *dst = g2d + (size_t)cidx[2 * p + (for_b ? 1 : 0)] * G2D_STRIDE;
              atomicAdd(dst + (even ? ((lane >> 1) & 7) : 8), even ? tot : tot8);
            }
          }
        }
        __syncthreads();  // cf, xidx and cidx reused by the next batch
        if (b >= 1) {
#pragma unroll
          for (int k = 0; k < PER; ++k) xidx[tid + k * NT] = mine[k];
        }
      }
    }
    __syncthreads();
  }
  if (COUNT) {
    atomicAdd(&counters[2], (unsigned long long)n_eval);
    atomicAdd(&counters[3], (unsigned long long)n_contrib);
    if (tid == 0) atomicAdd(&counters[5], n_staged);
  }
}

// Longest-first order of the backward's tiles: a tile's work is the largest number of list
// entries any of its pixels processed in the forward; tiles are ordered by the log2 class of
// that work, most first, so that the persistent CTAs start the long tiles early and the short
// ones fill in at the end. Any order gives the same gradients up to the order of their sums.
// The same launch zeroes the records' gradient accumulators (16-byte stores over the grid),
// which the backward rasterizer adds into next.
__global__ void __launch_bounds__(256)
    tile_work_kernel(const uint32_t *__restrict__ ranges, const uint32_t *__restrict__ n_processed,
                     Views vs, uint32_t *status, uint32_t *__restrict__ bucket,
                     uint32_t *__restrict__ hist, float4 *__restrict__ g2d4, int64_t n_g2d4) {
  __shared__ uint32_t s_hist[WORK_BUCKETS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < WORK_BUCKETS) s_hist[threadIdx.x] = 0u;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_g2d4;
       j += (int64_t)gridDim.x * blockDim.x)
    g2d4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * 8 + warp;
  if (t < vs.total_tiles) {
    const ListBounds bd = list_bounds(status);
    const TileInfo ti = tile_info(vs, t, ranges, bd, status);
    const View &V = vs.v[ti.v];
    const bool lists_ok = *(volatile const uint32_t *)status == 0u;
    uint32_t m = 0;
    const int px = ti.tx * TILE + (lane & (TILE - 1));
#pragma unroll
    for (int r = 0; r < TILE / 2; ++r) {
      const int py = ti.ty * TILE + 2 * r + (lane >> 4);
      if (px < V.width && py < V.height)
        m = max(m, __ldg(n_processed + V.pixel_offset + (int64_t)py * V.width + px));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    m = lists_ok ? min(m, ti.count) : 0u;
    const uint32_t b = min(32u - (uint32_t)__clz(m), (uint32_t)WORK_BUCKETS - 1u);
    if (lane == 0) {
      bucket[t] = b;
      atomicAdd(&s_hist[b], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x < WORK_BUCKETS && s_hist[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_hist[threadIdx.x]);
}

__global__ void __launch_bounds__(1024)
    tile_order_kernel(const uint32_t *__restrict__ bucket, const uint32_t *__restrict__ hist,
                      uint32_t *__restrict__ cursor, int64_t total_tiles,
                      uint32_t *__restrict__ order, uint32_t *status) {
  __shared__ uint32_t s_off[WORK_BUCKETS];
  if (threadIdx.x < 32) {  // start of each class: the tiles of all heavier classes come first
    const uint32_t h = hist[threadIdx.x];
    uint32_t x = h;  // suffix sum over the classes b' >= b
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_down_sync(0xffffffffu, x, o);
      if (threadIdx.x + o < 32) x += y;
    }
    s_off[threadIdx.x] = x - h;
  }
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = t < total_tiles;
  const uint32_t b = in ? bucket[t] : 0xffffffffu;
  // one atomic per (warp, class): lanes of the same class share the leader's claim
  const uint32_t peers = __match_any_sync(0xffffffffu, b);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (in && lane == leader) base = atomicAdd(&cursor[b], (uint32_t)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  const uint32_t slot = s_off[b & (WORK_BUCKETS - 1)] + base + __popc(peers & lanemask_lt());
  if (in && in_bounds(slot, (uint64_t)total_tiles, status)) order[slot] = (uint32_t)t;
}

template <typename K>
int occupancy_of(K kernel, int threads) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess) return 1;
  return occ > 0 ? occ : 1;
}

template <int PPT>
cudaError_t fwd_launch(const fgs_record *records, const uint32_t *vals, const uint32_t *ranges,
                       const Views &vs, float bg0, float bg1, float bg2, float *images,
                       float *final_T, uint32_t *n_processed, WsHeader *hdr, bool instrument,
                       cudaStream_t st) {
  constexpr int NT = TILE_PIX / PPT;
  static int occ = 0;
  if (occ == 0) occ = occupancy_of(raster_fwd_kernel<PPT, false>, NT);
  int64_t grid = (int64_t)sm_count() * occ;
  if (grid > vs.total_tiles) grid = vs.total_tiles;
  if (grid < 1) grid = 1;
  if (instrument)
    raster_fwd_kernel<PPT, true><<<(unsigned)grid, NT, 0, st>>>(
        records, vals, ranges, vs, bg0, bg1, bg2, images, final_T, n_processed,
        &hdr->raster_tiles, &hdr->status, hdr->counters);
  else
    raster_fwd_kernel<PPT, false><<<(unsigned)grid, NT, 0, st>>>(
        records, vals, ranges, vs, bg0, bg1, bg2, images, final_T, n_processed,
        &hdr->raster_tiles, &hdr->status, hdr->counters);
  return cudaGetLastError();
}

template <int PPT>
cudaError_t bwd_launch(const fgs_record *records, const uint32_t *vals, const uint32_t *ranges,
                       const Views &vs, float bg0, float bg1, float bg2, const float *final_T,
                       const uint32_t *n_processed, const float *dL, float *g2d,
                       const uint32_t *order, uint32_t *tile_counter, WsHeader *hdr,
                       bool instrument, cudaStream_t st) {
  constexpr int NT = TILE_PIX / PPT;
  static int occ = 0;
  if (occ == 0) occ = occupancy_of(raster_bwd_kernel<PPT, false>, NT);
  int64_t grid = (int64_t)sm_count() * occ;
  if (grid > vs.total_tiles) grid = vs.total_tiles;
  if (grid < 1) grid = 1;
  if (instrument)
    raster_bwd_kernel<PPT, true><<<(unsigned)grid, NT, 0, st>>>(
        records, vals, ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL, g2d, order,
        tile_counter, &hdr->status, hdr->counters);
  else
    raster_bwd_kernel<PPT, false><<<(unsigned)grid, NT, 0, st>>>(
        records, vals, ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL, g2d, order,
        tile_counter, &hdr->status, hdr->counters);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raster_fwd(const fgs_record *records, const uint32_t *vals,
                              const uint32_t *tile_ranges, const Views &vs, float bg0, float bg1,
                              float bg2, float *images, float *final_T, uint32_t *n_processed,
                              char *ws, const WsLayout &L, const CallOpts &opt,
                              cudaStream_t st) {
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.header);
  cudaError_t e = cudaMemsetAsync(&hdr->raster_tiles, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const bool ins = opt.instrument;
  if (opt.ev_before && (e = cudaEventRecord(opt.ev_before, st)) != cudaSuccess) return e;
  switch (opt.fwd_ppt) {
    case 2: e = fwd_launch<2>(records, vals, tile_ranges, vs, bg0, bg1, bg2, images, final_T, n_processed, hdr, ins, st); break;
    case 4: e = fwd_launch<4>(records, vals, tile_ranges, vs, bg0, bg1, bg2, images, final_T, n_processed, hdr, ins, st); break;
    default: e = fwd_launch<1>(records, vals, tile_ranges, vs, bg0, bg1, bg2, images, final_T, n_processed, hdr, ins, st); break;
  }
  if (e == cudaSuccess && opt.ev_after) e = cudaEventRecord(opt.ev_after, st);
  return e;
}

cudaError_t launch_raster_bwd(const fgs_record *records, const uint32_t *vals,
                              const uint32_t *tile_ranges, const Views &vs, float bg0, float bg1,
                              float bg2, const float *final_T, const uint32_t *n_processed,
                              const float *dL_dimages, int64_t n_records, char *ws,
                              const WsLayout &L, const CallOpts &opt, cudaStream_t st) {
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.header);
  float *g2d = reinterpret_cast<float *>(ws + L.g2d);
  uint32_t *order = reinterpret_cast<uint32_t *>(ws + L.tile_order);
  uint32_t *bucket = order + vs.total_tiles;
  // WORK_BUCKETS class counts, WORK_BUCKETS cursors, then the persistent CTAs' tile counter:
  // one memset clears the three
  uint32_t *hist = bucket + vs.total_tiles;
  uint32_t *tile_counter = hist + 2 * WORK_BUCKETS;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (2 * WORK_BUCKETS + 1), st);
  if (e != cudaSuccess) return e;
  const size_t g2d_bytes = sizeof(float) * G2D_STRIDE * (size_t)n_records;
  static_assert(G2D_STRIDE % 4 == 0, "gradient rows zeroed as float4");
  if (vs.total_tiles > 0) {
    // a warp per tile, and enough CTAs that each thread zeroes at most eight float4
    const int64_t n4 = (int64_t)(g2d_bytes / sizeof(float4));
    const int64_t blocks = std::max((vs.total_tiles + 7) / 8, (n4 + 2047) / 2048);
    tile_work_kernel<<<(unsigned)blocks, 256, 0, st>>>(tile_ranges, n_processed, vs, &hdr->status,
                                                       bucket, hist,
                                                       reinterpret_cast<float4 *>(g2d), n4);
    tile_order_kernel<<<(unsigned)((vs.total_tiles + 1023) / 1024), 1024, 0, st>>>(
        bucket, hist, hist + WORK_BUCKETS, vs.total_tiles, order, &hdr->status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if ((e = cudaMemsetAsync(g2d, 0, g2d_bytes, st)) != cudaSuccess) {
    return e;
  }
  const bool ins = opt.instrument;
  if (opt.ev_before && (e = cudaEventRecord(opt.ev_before, st)) != cudaSuccess) return e;
  switch (opt.bwd_ppt) {
    case 1: e = bwd_launch<1>(records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d, order, tile_counter, hdr, ins, st); break;
    case 2: e = bwd_launch<2>(records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d, order, tile_counter, hdr, ins, st); break;
    case 4: e = bwd_launch<4>(records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d, order, tile_counter, hdr, ins, st); break;
    default: e = bwd_launch<8>(records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d, order, tile_counter, hdr, ins, st); break;
  }
  if (e == cudaSuccess && opt.ev_after) e = cudaEventRecord(opt.ev_after, st);
  return e;
}

}  // namespace fgs
