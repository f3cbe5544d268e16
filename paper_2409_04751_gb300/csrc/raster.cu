// raster.cu - per-tile alpha blending (Sec. 3.1 "Rendering"; Sec. 4.1 renderCUDA) and its
// backward, sm_103a.
//
// One CTA per 16x16 tile with 256/PPT threads; each thread owns PPT vertically adjacent pixels
// (PPT = 1, 2 or 4, the "work shape"; the image does not depend on it). CTAs are persistent and
// take tiles from an atomic queue. Each tile's Gaussians are staged through shared memory in
// batches of 256 records: every thread issues TMA bulk copies (cp.async.bulk, 48 bytes each) of
// its share, completing on an mbarrier, and the next batch is in flight while the current one is
// blended (two stages). The sorted indices of the batch after next are prefetched into registers.
// A warp whose pixels have all stopped skips the batch (warp ballot); the CTA leaves the tile
// when all its pixels have stopped.
//
// The backward replays each pixel's blend back to front from its final transmittance and the
// number of list entries it processed (both written by the forward), recovering the
// transmittance before each Gaussian by division; nothing per (pixel, Gaussian) is stored. Per
// contributing pair it accumulates nine sums that depend on the pixel only: the moments
// sum dL/dp (dx, dy, dx^2, dx dy, dy^2) of the exponent p = -0.5 d^T conic d, sum dL/dalpha
// alpha_raw, and dL/drgb. Each thread first sums its own pixels; the warp then reduces the nine
// sums with a transpose reduction (each exchange halves the values a lane carries: 14 shuffles
// instead of 45) and eight lanes add their totals to the record's accumulator. The preprocess
// backward turns the moments into dL/dxy, dL/dconic and dL/dopacity with the record's conic and
// opacity.
#include "fgs_internal.cuh"

namespace fgs {

namespace {

constexpr int TILE_PIX = TILE * TILE;  // 256 pixels per tile
// Gaussians per staged batch: 256, or 128 for the 4-pixels-per-thread shape, whose CTAs are
// small and need a small shared-memory footprint to keep enough of them resident
template <int PPT>
struct Batch {
  static constexpr int N = PPT == 8 ? 64 : (PPT == 4 ? 128 : 256);
};
constexpr uint32_t REC_BYTES = sizeof(fgs_record);
static_assert(REC_BYTES == 48, "record size");

struct TileInfo {
  int v;
  int tx, ty;
  uint32_t start, count;
};

__device__ __forceinline__ TileInfo tile_info(const Views &vs, int64_t t,
                                              const uint32_t *__restrict__ ranges) {
  TileInfo ti;
  ti.v = view_of_tile(vs, t);
  const View &V = vs.v[ti.v];
  const int64_t local = t - V.tile_offset;
  ti.ty = (int)(local / V.tiles_x);
  ti.tx = (int)(local - (int64_t)ti.ty * V.tiles_x);
  const uint2 rg = __ldg(reinterpret_cast<const uint2 *>(ranges) + t);
  ti.start = rg.x;
  ti.count = rg.y > rg.x ? rg.y - rg.x : 0u;
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
                                         uint32_t lo, uint32_t cnt, uint32_t (&idx)[PER]) {
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const uint32_t slot = threadIdx.x + k * NT;
    idx[k] = slot < cnt ? __ldg(vals + base + lo + slot) : 0u;
  }
}


// The exponent of the blend in base 2, e = A' dx^2 + B' dx dy + C' dy^2 + log2(opacity) with
// (dx, dy) = pixel centre - mean, A' = -log2(e) conic_xx / 2, B' = -log2(e) conic_xy,
// C' = -log2(e) conic_yy / 2, written in tile-centred pixel coordinates (u, v) = pixel centre
// - tile centre: e = K0 + Kx u + Ky v + A' u^2 + B' u v + C' v^2 (five FMAs per pixel; with
// |u|, |v| <= 7.5 the terms stay small, so rounding stays near that of the direct form). The
// forward (every work shape) and the backward evaluate it the same way, so they take the same
// alpha >= 1/255 decisions. xf[0] = (K0, Kx, Ky, A'), xf[1] = (B', C', r, g),
// xf[2] = (b, mean - tile centre offsets cx, cy, 0) with dx = u + cx, dy = v + cy.
__device__ __forceinline__ void stage_record(const fgs_record &g, float tile_cx, float tile_cy,
                                             float4 *xf) {
  const float A = -0.5f * LOG2E * g.conic[0], B = -LOG2E * g.conic[1];
  const float C = -0.5f * LOG2E * g.conic[2], lo2o = log2f(g.opacity);
  const float cx = tile_cx - g.xy[0], cy = tile_cy - g.xy[1];
  const float K0 = fmaf(cx, fmaf(A, cx, B * cy), fmaf(C * cy, cy, lo2o));
  const float Kx = fmaf(2.f * A, cx, B * cy), Ky = fmaf(B, cx, 2.f * C * cy);
  xf[0] = make_float4(K0, Kx, Ky, A);
  xf[1] = make_float4(B, C, g.rgb[0], g.rgb[1]);
  xf[2] = make_float4(g.rgb[2], cx, cy, 0.f);
}

__device__ __forceinline__ float exponent(const float4 &a, const float4 &c, float u, float v,
                                          float uu, float uv, float vv) {
  return fmaf(uu, a.w, fmaf(uv, c.x, fmaf(vv, c.y, fmaf(v, a.z, fmaf(u, a.y, a.x)))));
}

template <int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE_PIX / PPT, PPT == 1 ? 5 : 1)
    raster_fwd_kernel(const fgs_record *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ ranges, Views vs, float bg0, float bg1,
                      float bg2, float *__restrict__ images, float *__restrict__ final_T,
                      uint32_t *__restrict__ n_processed, uint32_t *tile_counter,
                      uint32_t *status, unsigned long long *counters) {
  constexpr int NT = TILE_PIX / PPT;
  constexpr int BATCH = Batch<PPT>::N;
  constexpr int PER = BATCH / NT;  // copies each thread issues per batch
  __shared__ __align__(128) fgs_record raw[2][BATCH];
  __shared__ __align__(16) float4 xf[BATCH][3];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_tile;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], NT);
    mbar_init(&bar[1], NT);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase0 = 0, phase1 = 0;
  uint32_t n_eval = 0, n_blend = 0;
  const int lx = tid & (TILE - 1), ly0 = (tid / TILE) * PPT;
  // after a device-side error in the binning the lists are undefined: render background only
  const bool lists_ok = *(volatile const uint32_t *)status == 0u;

  for (;;) {
    if (tid == 0) s_tile = (int64_t)atomicAdd(tile_counter, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    __syncthreads();
    if (t >= vs.total_tiles) break;
    const TileInfo ti = tile_info(vs, t, ranges);
    const View &V = vs.v[ti.v];
    const int px = ti.tx * TILE + lx;
    // tile centre (between pixel centres 7 and 8) and this pixel's offset from it
    const float tile_cx = (float)(ti.tx * TILE) + 0.5f * TILE, tile_cy = (float)(ti.ty * TILE) + 0.5f * TILE;
    const float fu = (float)lx - 7.5f, fv = (float)ly0 - 7.5f;
    const float uu = fu * fu, uv = fu * fv, vv = fv * fv;
    float fpy[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
    uint32_t last[PPT];
    bool live[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = ti.ty * TILE + ly0 + k;
      fpy[k] = (float)py + 0.5f;
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
      load_idx<NT, PER>(vals, ti.start, 0, count, idx);
      load_idx<NT, PER>(vals, ti.start, BATCH, count > BATCH ? count - BATCH : 0u, idx_next);
      fence_proxy_async_smem();
      issue_batch<NT, PER>(raw[0], &bar[0], rec, idx, min(count, (uint32_t)BATCH));
      for (uint32_t b = 0; b < nb; ++b) {
        const int s = b & 1;
        const uint32_t lo = b * BATCH;
        const uint32_t cnt = min((uint32_t)BATCH, count - lo);
        if (b + 1 < nb) {
          fence_proxy_async_smem();
          issue_batch<NT, PER>(raw[s ^ 1], &bar[s ^ 1], rec, idx_next,
                               min((uint32_t)BATCH, count - lo - BATCH));
          const uint32_t lo2 = lo + 2 * BATCH;
          load_idx<NT, PER>(vals, ti.start, lo2, count > lo2 ? count - lo2 : 0u, idx_next);
        }
        const bool ok = mbar_wait(&bar[s], s ? phase1 : phase0, status);
        if (s) phase1 ^= 1u; else phase0 ^= 1u;
        if (__syncthreads_or(!ok)) {  // a copy never landed: drain (bounded) and leave
          if (b + 1 < nb) mbar_wait(&bar[s ^ 1], s ? phase0 : phase1, status);
          return;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const uint32_t slot = tid + k * NT;
          if (slot < cnt) {
            stage_record(raw[s][slot], tile_cx, tile_cy, xf[slot]);
          }
        }
        __syncthreads();
        if (PPT == 1 && !__all_sync(0xffffffffu, done)) {
          // one pixel per thread, two list entries per iteration
          const uint32_t lo1 = lo + 1;
          if (!done) {
            bool stop = false;
            uint32_t j = 0;
            for (; j < cnt; j += 2) {
              const bool two = j + 1 < cnt;
              const float4 a0 = xf[j][0], c0 = xf[j][1];
              const uint32_t j1 = two ? j + 1 : j;
              const float4 a1 = xf[j1][0], c1 = xf[j1][1];
              const float e0 = exponent(a0, c0, fu, fv, uu, uv, vv);
              const float e1 = exponent(a1, c1, fu, fv, uu, uv, vv);
              if (COUNT) ++n_eval;
              if (e0 >= LOG2_ALPHA_MIN) {
                const float alpha = fminf(ALPHA_MAX, ex2_approx(e0));
                const float Tn = fmaf(-alpha, T[0], T[0]);
                if (Tn < T_MIN) {
                  stop = true;
                  break;
                }
                const float wgt = alpha * T[0];
                C0[0] = fmaf(c0.z, wgt, C0[0]);
                C1[0] = fmaf(c0.w, wgt, C1[0]);
                C2[0] = fmaf(xf[j][2].x, wgt, C2[0]);
                T[0] = Tn;
                last[0] = lo1 + j;
                if (COUNT) ++n_blend;
              }
              if (!two) break;
              if (COUNT) ++n_eval;
              if (e1 >= LOG2_ALPHA_MIN) {
                const float alpha = fminf(ALPHA_MAX, ex2_approx(e1));
                const float Tn = fmaf(-alpha, T[0], T[0]);
                if (Tn < T_MIN) {
                  stop = true;
                  break;
                }
                const float wgt = alpha * T[0];
                C0[0] = fmaf(c1.z, wgt, C0[0]);
                C1[0] = fmaf(c1.w, wgt, C1[0]);
                C2[0] = fmaf(xf[j1][2].x, wgt, C2[0]);
                T[0] = Tn;
                last[0] = lo1 + j1;
                if (COUNT) ++n_blend;
              }
            }
            if (stop) live[0] = false;
            done = !live[0];
          }
        } else if (!__all_sync(0xffffffffu, done)) {
          const uint32_t lo1 = lo + 1;
          for (uint32_t j = 0; j < cnt && !done; ++j) {
            const float4 a = xf[j][0];
            const float4 c = xf[j][1];
            {
              bool any_live = false;
#pragma unroll
              for (int k = 0; k < PPT; ++k) {
                if (live[k]) {
                  const float v = fv + (float)k;
                  const float e = exponent(a, c, fu, v, uu, fu * v, v * v);
                  if (COUNT) ++n_eval;
                  if (e >= LOG2_ALPHA_MIN) {
                    const float alpha = fminf(ALPHA_MAX, ex2_approx(e));
                    const float Tn = fmaf(-alpha, T[k], T[k]);
                    if (Tn < T_MIN) {
                      live[k] = false;
                    } else {
                      const float wgt = alpha * T[k];
                      C0[k] = fmaf(c.z, wgt, C0[k]);
                      C1[k] = fmaf(c.w, wgt, C1[k]);
                      C2[k] = fmaf(xf[j][2].x, wgt, C2[k]);
                      T[k] = Tn;
                      last[k] = lo1 + j;
                      if (COUNT) ++n_blend;
                    }
                  }
                }
                any_live = any_live || live[k];
              }
              if (!any_live) break;
            }
          }
          bool any_live = false;
#pragma unroll
          for (int k = 0; k < PPT; ++k) any_live = any_live || live[k];
          done = !any_live;
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
  }
}

// Warp sum of eight values by transpose reduction: at each exchange a lane keeps half of its
// values and sends the other half to its partner, so 4 + 2 + 1 + 1 + 1 shuffles reduce all
// eight. On return lane l holds the total of value 4*b4 + 2*b3 + b2 (b_i = bit i of l).
__device__ __forceinline__ float warp_transpose_sum8(const float (&a)[8], int lane) {
  float b[4], c[2];
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float keep = h4 ? a[k + 4] : a[k];
    const float send = h4 ? a[k] : a[k + 4];
    b[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float keep = h3 ? b[k + 2] : b[k];
    const float send = h3 ? b[k] : b[k + 2];
    c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float d = (h2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h2 ? c[0] : c[1], 4);
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE_PIX / PPT)
    raster_bwd_kernel(const fgs_record *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ ranges, Views vs, float bg0, float bg1,
                      float bg2, const float *__restrict__ final_T,
                      const uint32_t *__restrict__ n_processed, const float *__restrict__ dLdimg,
                      float *__restrict__ g2d, uint32_t *tile_counter, uint32_t *status,
                      unsigned long long *counters) {
  constexpr int NT = TILE_PIX / PPT;
  constexpr int BATCH = Batch<PPT>::N;
  constexpr int PER = BATCH / NT;
  __shared__ __align__(128) fgs_record raw[2][BATCH];
  __shared__ __align__(16) float4 xf[BATCH][3];
  __shared__ uint32_t xidx[BATCH];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_tile;
  __shared__ uint32_t s_max;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar[0], NT);
    mbar_init(&bar[1], NT);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase0 = 0, phase1 = 0;
  uint32_t n_eval = 0, n_contrib = 0;
  const int lx = tid & (TILE - 1), ly0 = (tid / TILE) * PPT;
  // after a device-side error in the binning the lists are undefined: no gradient flows
  const bool lists_ok = *(volatile const uint32_t *)status == 0u;

  for (;;) {
    if (tid == 0) {
      s_tile = (int64_t)atomicAdd(tile_counter, 1u);
      s_max = 0u;
    }
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= vs.total_tiles) break;
    const TileInfo ti = tile_info(vs, t, ranges);
    const View &V = vs.v[ti.v];
    const int px = ti.tx * TILE + lx;
    const float tile_cx = (float)(ti.tx * TILE) + 0.5f * TILE, tile_cy = (float)(ti.ty * TILE) + 0.5f * TILE;
    const float fu = (float)lx - 7.5f, fv = (float)ly0 - 7.5f, uu = fu * fu;
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
        load_idx<NT, PER>(vals, ti.start, lo0, max_last - lo0, idx);
        if (nb >= 2) load_idx<NT, PER>(vals, ti.start, lo0 - BATCH, BATCH, idx_next);
        fence_proxy_async_smem();
        issue_batch<NT, PER>(raw[0], &bar[0], rec, idx, max_last - lo0);
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
#pragma unroll
          for (int k = 0; k < PER; ++k) mine[k] = idx_next[k];
          if (b >= 2) load_idx<NT, PER>(vals, ti.start, lo - 2 * BATCH, BATCH, idx_next);
        }
        const bool ok = mbar_wait(&bar[s], s ? phase1 : phase0, status);
        if (s) phase1 ^= 1u; else phase0 ^= 1u;
        if (__syncthreads_or(!ok)) {  // a copy never landed: drain (bounded) and leave
          if (b >= 1) mbar_wait(&bar[s ^ 1], s ? phase0 : phase1, status);
          return;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const uint32_t slot = tid + k * NT;
          if (slot < cnt) {
            stage_record(raw[s][slot], tile_cx, tile_cy, xf[slot]);
          }
        }
        __syncthreads();
        for (int j = (int)cnt - 1; j >= 0; --j) {
          const uint32_t pos = lo + (uint32_t)j;
          const bool any_pos = pos < my_max;
          if (!__any_sync(0xffffffffu, any_pos)) continue;
          float v[9];
#pragma unroll
          for (int q = 0; q < 9; ++q) v[q] = 0.f;
          bool contrib = false;
          if (any_pos) {
            const float4 a = xf[j][0];
            const float4 c = xf[j][1];
            const float4 c2 = xf[j][2];
            const float dx = fu + c2.y;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
              if (pos < last[k]) {
                const float vk = fv + (float)k;
                const float e = exponent(a, c, fu, vk, uu, fu * vk, vk * vk);
                const float dy = vk + c2.z;
                if (COUNT) ++n_eval;
                if (e >= LOG2_ALPHA_MIN) {
                  contrib = true;
                  if (COUNT) ++n_contrib;
                  const float cb = c2.x;
                  const float araw = ex2_approx(e);
                  const float alpha = fminf(ALPHA_MAX, araw);
                  const float om = rcp_approx(1.f - alpha);
                  T[k] *= om;  // transmittance before this Gaussian
                  const float wgt = alpha * T[k];
                  const float gc = G0[k] * c.z + G1[k] * c.w + G2[k] * cb;  // <dL/dC, colour>
                  // dL/dalpha = <dL/dC, colour T - behind / (1 - alpha)>
                  const float dLda = fmaf(T[k], gc, -om * GS[k]);
                  GS[k] = fmaf(gc, wgt, GS[k]);
                  v[6] = fmaf(G0[k], wgt, v[6]);
                  v[7] = fmaf(G1[k], wgt, v[7]);
                  v[8] = fmaf(G2[k], wgt, v[8]);
                  if (araw < ALPHA_MAX) {
                    // alpha = opacity exp(p), p = -0.5 d^T conic d: accumulate the moments of
                    // dL/dp over the pixel offsets; the conic and opacity are applied once per
                    // record in the preprocess backward
                    const float dLdp = dLda * alpha;
                    const float tx = dLdp * dx, ty = dLdp * dy;
                    v[0] += tx;
                    v[1] += ty;
                    v[2] = fmaf(tx, dx, v[2]);
                    v[3] = fmaf(tx, dy, v[3]);
                    v[4] = fmaf(ty, dy, v[4]);
                    v[5] = fmaf(dLda, araw, v[5]);
                  }
                }
              }
            }
          }
          if (__any_sync(0xffffffffu, contrib)) {
            const float a8[8] = {v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]};
            const float tot = warp_transpose_sum8(a8, lane);
            const float tot8 = warp_sum(v[8]);
            float *dst = g2d + (size_t)xidx[j] * G2D_STRIDE;
            if ((lane & 3) == 0) atomicAdd(dst + (lane >> 2), tot);
            if (lane == 0) atomicAdd(dst + 8, tot8);
          }
        }
        __syncthreads();  // xf / xidx reused by the next batch
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
  }
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
                       float *final_T, uint32_t *n_processed, WsHeader *hdr, cudaStream_t st) {
  constexpr int NT = TILE_PIX / PPT;
  static int occ = 0;
  if (occ == 0) occ = occupancy_of(raster_fwd_kernel<PPT, false>, NT);
  int64_t grid = (int64_t)sm_count() * occ;
  if (grid > vs.total_tiles) grid = vs.total_tiles;
  if (grid < 1) grid = 1;
  if (instrumented())
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
                       const uint32_t *n_processed, const float *dL, float *g2d, WsHeader *hdr,
                       cudaStream_t st) {
  constexpr int NT = TILE_PIX / PPT;
  static int occ = 0;
  if (occ == 0) occ = occupancy_of(raster_bwd_kernel<PPT, false>, NT);
  int64_t grid = (int64_t)sm_count() * occ;
  if (grid > vs.total_tiles) grid = vs.total_tiles;
  if (grid < 1) grid = 1;
  if (instrumented())
    raster_bwd_kernel<PPT, true><<<(unsigned)grid, NT, 0, st>>>(
        records, vals, ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL, g2d,
        &hdr->backward_tiles, &hdr->status, hdr->counters);
  else
    raster_bwd_kernel<PPT, false><<<(unsigned)grid, NT, 0, st>>>(
        records, vals, ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL, g2d,
        &hdr->backward_tiles, &hdr->status, hdr->counters);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raster_fwd(const fgs_record *records, const uint32_t *vals,
                              const uint32_t *tile_ranges, const Views &vs, float bg0, float bg1,
                              float bg2, float *images, float *final_T, uint32_t *n_processed,
                              char *ws, const WsLayout &L, cudaStream_t st) {
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.header);
  cudaError_t e = cudaMemsetAsync(&hdr->raster_tiles, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  switch (raster_shape(0)) {
    case 1: return fwd_launch<1>(records, vals, tile_ranges, vs, bg0, bg1, bg2, images, final_T, n_processed, hdr, st);
    case 4: return fwd_launch<4>(records, vals, tile_ranges, vs, bg0, bg1, bg2, images, final_T, n_processed, hdr, st);
    default: return fwd_launch<2>(records, vals, tile_ranges, vs, bg0, bg1, bg2, images, final_T, n_processed, hdr, st);
  }
}

cudaError_t launch_raster_bwd(const fgs_record *records, const uint32_t *vals,
                              const uint32_t *tile_ranges, const Views &vs, float bg0, float bg1,
                              float bg2, const float *final_T, const uint32_t *n_processed,
                              const float *dL_dimages, int64_t n_records, char *ws,
                              const WsLayout &L, cudaStream_t st) {
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.header);
  float *g2d = reinterpret_cast<float *>(ws + L.g2d);
  cudaError_t e = cudaMemsetAsync(&hdr->backward_tiles, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(g2d, 0, sizeof(float) * G2D_STRIDE * (size_t)n_records, st)) != cudaSuccess)
    return e;
  switch (raster_shape(1)) {
    case 1: return bwd_launch<1>(records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d, hdr, st);
    case 8: return bwd_launch<8>(records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d, hdr, st);
    case 4: return bwd_launch<4>(records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d, hdr, st);
    default: return bwd_launch<2>(records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d, hdr, st);
  }
}

}  // namespace fgs
