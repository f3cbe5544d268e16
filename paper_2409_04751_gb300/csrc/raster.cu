// raster.cu - per-tile alpha blending (Sec. 3.1 "Rendering"; Sec. 4.1 renderCUDA) and its
// backward, sm_103a.
//
// One CTA of 256 threads per 16x16 tile, one pixel per thread; CTAs are persistent and take
// tiles from an atomic queue. Each tile's Gaussians are staged through shared memory in batches
// of 256: every thread issues one TMA bulk copy (cp.async.bulk, 48 bytes) of its record,
// completing on an mbarrier, and the next batch is in flight while the current one is blended
// (two stages). The sorted indices of the batch after next are prefetched into registers. A
// warp whose pixels have all stopped skips the batch (warp ballot); the CTA leaves the tile
// when all 256 pixels have stopped.
//
// The backward replays each pixel's blend back to front from its final transmittance and the
// number of list entries it processed (both written by the forward), recovering the
// transmittance before each Gaussian by division; nothing per (pixel, Gaussian) is stored.
// Screen-space gradients are summed over the warp with shuffles and added to the record's
// accumulator with one vector atomic per warp.
#include "fgs_internal.cuh"

namespace fgs {

namespace {

constexpr int RT = 256;     // threads per tile CTA (one per pixel)
constexpr int BATCH = 256;  // Gaussians per staged batch
constexpr uint32_t REC_BYTES = sizeof(fgs_record);
static_assert(REC_BYTES == 48, "record size");

struct TileInfo {
  int64_t t;
  int v;
  int px, py;
  bool inside;
  uint32_t start, count;
};

__device__ __forceinline__ TileInfo tile_info(const Views &vs, int64_t t,
                                              const uint32_t *__restrict__ ranges) {
  TileInfo ti;
  ti.t = t;
  ti.v = view_of_tile(vs, t);
  const View &V = vs.v[ti.v];
  const int64_t local = t - V.tile_offset;
  const int ty = (int)(local / V.tiles_x), tx = (int)(local - (int64_t)ty * V.tiles_x);
  ti.px = tx * TILE + (threadIdx.x & (TILE - 1));
  ti.py = ty * TILE + (threadIdx.x / TILE);
  ti.inside = ti.px < V.width && ti.py < V.height;
  const uint2 rg = __ldg(reinterpret_cast<const uint2 *>(ranges) + t);
  ti.start = rg.x;
  ti.count = rg.y > rg.x ? rg.y - rg.x : 0u;
  return ti;
}

// Issue this thread's share of a batch: one 48-byte bulk copy of its record, or a plain
// arrival when the batch has no entry for it. The barrier expects RT arrivals per phase.
__device__ __forceinline__ void issue_batch(fgs_record *stage, uint64_t *bar,
                                            const fgs_record *__restrict__ rec, uint32_t idx,
                                            bool has) {
  if (has) {
    mbar_arrive_expect_tx(bar, REC_BYTES);
    bulk_g2s(stage + threadIdx.x, rec + idx, REC_BYTES, bar);
  } else {
    mbar_arrive(bar);
  }
}

template <bool COUNT>
__global__ void __launch_bounds__(RT)
    raster_fwd_kernel(const fgs_record *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ ranges, Views vs, float bg0, float bg1,
                      float bg2, float *__restrict__ images, float *__restrict__ final_T,
                      uint32_t *__restrict__ n_processed, uint32_t *tile_counter,
                      uint32_t *status, unsigned long long *counters) {
  __shared__ __align__(128) fgs_record raw[2][BATCH];
  __shared__ __align__(16) float4 xf[BATCH][3];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_tile;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], RT);
    mbar_init(&bar[1], RT);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase0 = 0, phase1 = 0;
  uint32_t n_eval = 0, n_blend = 0;

  for (;;) {
    if (tid == 0) s_tile = (int64_t)atomicAdd(tile_counter, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    __syncthreads();
    if (t >= vs.total_tiles) break;
    const TileInfo ti = tile_info(vs, t, ranges);
    const View &V = vs.v[ti.v];
    const float fpx = (float)ti.px + 0.5f, fpy = (float)ti.py + 0.5f;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !ti.inside;
    const uint32_t count = ti.count;
    const uint32_t nb = (count + BATCH - 1) / BATCH;

    if (nb > 0) {
      uint32_t idx_next = 0;
      {
        const bool has0 = (uint32_t)tid < count;
        const uint32_t idx0 = has0 ? __ldg(vals + ti.start + tid) : 0u;
        if (BATCH + (uint32_t)tid < count) idx_next = __ldg(vals + ti.start + BATCH + tid);
        fence_proxy_async_smem();
        issue_batch(raw[0], &bar[0], rec, idx0, has0);
      }
      for (uint32_t b = 0; b < nb; ++b) {
        const int s = b & 1;
        const uint32_t cnt = min((uint32_t)BATCH, count - b * BATCH);
        if (b + 1 < nb) {
          const bool has = (b + 1) * BATCH + (uint32_t)tid < count;
          fence_proxy_async_smem();
          issue_batch(raw[s ^ 1], &bar[s ^ 1], rec, idx_next, has);
          const uint32_t q = (b + 2) * BATCH + (uint32_t)tid;
          idx_next = q < count ? __ldg(vals + ti.start + q) : 0u;
        }
        const bool ok = mbar_wait(&bar[s], s ? phase1 : phase0, status);
        if (s) phase1 ^= 1u; else phase0 ^= 1u;
        if (__syncthreads_or(!ok)) {  // a copy never landed: drain (bounded) and leave
          if (b + 1 < nb) mbar_wait(&bar[s ^ 1], s ? phase0 : phase1, status);
          return;
        }
        if ((uint32_t)tid < cnt) {
          const fgs_record &g = raw[s][tid];
          // exponent in base 2: e = A' dx^2 + B' dx dy + C' dy^2 + log2(opacity)
          xf[tid][0] = make_float4(g.xy[0], g.xy[1], -0.5f * LOG2E * g.conic[0], -LOG2E * g.conic[1]);
          xf[tid][1] = make_float4(-0.5f * LOG2E * g.conic[2], log2f(g.opacity), g.rgb[0], g.rgb[1]);
          xf[tid][2] = make_float4(g.rgb[2], 0.f, 0.f, 0.f);
        }
        __syncthreads();
        if (!__all_sync(0xffffffffu, done)) {
          for (uint32_t j = 0; j < cnt && !done; ++j) {
            const float4 a = xf[j][0];
            const float4 c = xf[j][1];
            const float dx = fpx - a.x, dy = fpy - a.y;
            const float e = fmaf(dx, fmaf(a.z, dx, a.w * dy), fmaf(c.x * dy, dy, c.y));
            if (COUNT) ++n_eval;
            if (e < LOG2_ALPHA_MIN) continue;
            const float alpha = fminf(ALPHA_MAX, exp2f(e));
            const float Tn = T * (1.f - alpha);
            if (Tn < T_MIN) {
              done = true;
              break;
            }
            const float wgt = alpha * T;
            C0 = fmaf(c.z, wgt, C0);
            C1 = fmaf(c.w, wgt, C1);
            C2 = fmaf(xf[j][2].x, wgt, C2);
            T = Tn;
            last = b * BATCH + j + 1;
            if (COUNT) ++n_blend;
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
    if (ti.inside) {
      const int64_t p = V.pixel_offset + (int64_t)ti.py * V.width + ti.px;
      const int64_t plane = (int64_t)V.width * V.height;
      float *img = images + 3 * V.pixel_offset + (int64_t)ti.py * V.width + ti.px;
      img[0] = fmaf(T, bg0, C0);
      img[plane] = fmaf(T, bg1, C1);
      img[2 * plane] = fmaf(T, bg2, C2);
      final_T[p] = T;
      n_processed[p] = last;
    }
  }
  if (COUNT) {
    atomicAdd(&counters[0], (unsigned long long)n_eval);
    atomicAdd(&counters[1], (unsigned long long)n_blend);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool COUNT>
__global__ void __launch_bounds__(RT)
    raster_bwd_kernel(const fgs_record *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ ranges, Views vs, float bg0, float bg1,
                      float bg2, const float *__restrict__ final_T,
                      const uint32_t *__restrict__ n_processed, const float *__restrict__ dLdimg,
                      float *__restrict__ g2d, uint32_t *tile_counter, uint32_t *status,
                      unsigned long long *counters) {
  __shared__ __align__(128) fgs_record raw[2][BATCH];
  __shared__ __align__(16) float4 xf[BATCH][4];
  __shared__ uint32_t xidx[BATCH];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_tile;
  __shared__ uint32_t s_max;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar[0], RT);
    mbar_init(&bar[1], RT);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase0 = 0, phase1 = 0;
  uint32_t n_eval = 0, n_contrib = 0;

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
    const float fpx = (float)ti.px + 0.5f, fpy = (float)ti.py + 0.5f;
    float T = 1.f, G0 = 0.f, G1 = 0.f, G2 = 0.f;
    uint32_t last = 0;
    if (ti.inside) {
      const int64_t p = V.pixel_offset + (int64_t)ti.py * V.width + ti.px;
      const int64_t plane = (int64_t)V.width * V.height;
      const float *gi = dLdimg + 3 * V.pixel_offset + (int64_t)ti.py * V.width + ti.px;
      T = final_T[p];
      last = min(n_processed[p], ti.count);
      G0 = gi[0]; G1 = gi[plane]; G2 = gi[2 * plane];
      atomicMax(&s_max, last);
    }
    // colour behind the current entry: sum over later blended entries + T_final bg
    float S0 = T * bg0, S1 = T * bg1, S2 = T * bg2;
    __syncthreads();
    const uint32_t max_last = s_max;
    const uint32_t nb = (max_last + BATCH - 1) / BATCH;

    if (nb > 0) {
      // batches from the back: it = 0 handles batch nb-1
      uint32_t idx_next = 0;
      {
        const uint32_t b0 = nb - 1;
        const bool has0 = b0 * BATCH + (uint32_t)tid < max_last;
        const uint32_t idx0 = has0 ? __ldg(vals + ti.start + b0 * BATCH + tid) : 0u;
        if (nb >= 2) idx_next = __ldg(vals + ti.start + (nb - 2) * BATCH + tid);
        fence_proxy_async_smem();
        issue_batch(raw[0], &bar[0], rec, idx0, has0);
        if (has0) xidx[tid] = idx0;
      }
      for (uint32_t it = 0; it < nb; ++it) {
        const uint32_t b = nb - 1 - it;
        const int s = it & 1;
        const uint32_t lo = b * BATCH;
        const uint32_t cnt = min((uint32_t)BATCH, max_last - lo);
        uint32_t my_idx = 0;
        if (b >= 1) {
          fence_proxy_async_smem();
          issue_batch(raw[s ^ 1], &bar[s ^ 1], rec, idx_next, true);
          my_idx = idx_next;
          idx_next = b >= 2 ? __ldg(vals + ti.start + (b - 2) * BATCH + tid) : 0u;
        }
        const bool ok = mbar_wait(&bar[s], s ? phase1 : phase0, status);
        if (s) phase1 ^= 1u; else phase0 ^= 1u;
        if (__syncthreads_or(!ok)) {  // a copy never landed: drain (bounded) and leave
          if (b >= 1) mbar_wait(&bar[s ^ 1], s ? phase0 : phase1, status);
          return;
        }
        if ((uint32_t)tid < cnt) {
          const fgs_record &g = raw[s][tid];
          xf[tid][0] = make_float4(g.xy[0], g.xy[1], -0.5f * LOG2E * g.conic[0], -LOG2E * g.conic[1]);
          xf[tid][1] = make_float4(-0.5f * LOG2E * g.conic[2], log2f(g.opacity), g.rgb[0], g.rgb[1]);
          xf[tid][2] = make_float4(g.rgb[2], g.conic[0], g.conic[1], g.conic[2]);
          xf[tid][3] = make_float4(g.opacity, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        for (int j = (int)cnt - 1; j >= 0; --j) {
          const uint32_t pos = lo + (uint32_t)j;
          float v[9];
          bool contrib = false;
          if (pos < last) {
            const float4 a = xf[j][0];
            const float4 c = xf[j][1];
            const float dx = fpx - a.x, dy = fpy - a.y;
            const float e = fmaf(dx, fmaf(a.z, dx, a.w * dy), fmaf(c.x * dy, dy, c.y));
            if (COUNT) ++n_eval;
            if (e >= LOG2_ALPHA_MIN) {
              contrib = true;
              if (COUNT) ++n_contrib;
              const float4 r2 = xf[j][2];
              const float araw = exp2f(e);
              const float alpha = fminf(ALPHA_MAX, araw);
              const float om = 1.f / (1.f - alpha);
              T *= om;  // transmittance before this Gaussian
              const float wgt = alpha * T;
              const float dLda = G0 * (c.z * T - S0 * om) + G1 * (c.w * T - S1 * om) +
                                 G2 * (r2.x * T - S2 * om);
              S0 = fmaf(c.z, wgt, S0);
              S1 = fmaf(c.w, wgt, S1);
              S2 = fmaf(r2.x, wgt, S2);
              v[6] = G0 * wgt; v[7] = G1 * wgt; v[8] = G2 * wgt;
              if (araw < ALPHA_MAX) {
                const float dLdp = dLda * alpha;  // p = -0.5 d^T conic d
                v[0] = dLdp * (r2.y * dx + r2.z * dy);
                v[1] = dLdp * (r2.z * dx + r2.w * dy);
                v[2] = -0.5f * dx * dx * dLdp;
                v[3] = -dx * dy * dLdp;
                v[4] = -0.5f * dy * dy * dLdp;
                v[5] = dLda * araw / xf[j][3].x;
              } else {
                v[0] = v[1] = v[2] = v[3] = v[4] = v[5] = 0.f;
              }
            }
          }
          if (__any_sync(0xffffffffu, contrib)) {
            if (!contrib) {
#pragma unroll
              for (int k = 0; k < 9; ++k) v[k] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) v[k] = warp_sum(v[k]);
            if (lane == 0) {
              float *dst = g2d + (size_t)xidx[j] * G2D_STRIDE;
              atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(v[0], v[1], v[2], v[3]));
              atomicAdd(reinterpret_cast<float4 *>(dst) + 1, make_float4(v[4], v[5], v[6], v[7]));
              atomicAdd(dst + 8, v[8]);
            }
          }
        }
        __syncthreads();  // xf / xidx reused by the next batch
        if (b >= 1) xidx[tid] = my_idx;
      }
    }
    __syncthreads();
  }
  if (COUNT) {
    atomicAdd(&counters[2], (unsigned long long)n_eval);
    atomicAdd(&counters[3], (unsigned long long)n_contrib);
  }
}

int g_fwd_occ = 0, g_bwd_occ = 0;

}  // namespace

cudaError_t launch_raster_fwd(const fgs_record *records, const uint32_t *vals,
                              const uint32_t *tile_ranges, const Views &vs, float bg0, float bg1,
                              float bg2, float *images, float *final_T, uint32_t *n_processed,
                              char *ws, const WsLayout &L, cudaStream_t st) {
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.header);
  cudaError_t e = cudaMemsetAsync(&hdr->raster_tiles, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (g_fwd_occ == 0) {
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, raster_fwd_kernel<false>, RT, 0)) != cudaSuccess)
      return e;
    g_fwd_occ = occ > 0 ? occ : 1;
  }
  int64_t grid = (int64_t)sm_count() * g_fwd_occ;
  if (grid > vs.total_tiles) grid = vs.total_tiles;
  if (grid < 1) grid = 1;
  if (instrumented())
    raster_fwd_kernel<true><<<(unsigned)grid, RT, 0, st>>>(
        records, vals, tile_ranges, vs, bg0, bg1, bg2, images, final_T, n_processed,
        &hdr->raster_tiles, &hdr->status, hdr->counters);
  else
    raster_fwd_kernel<false><<<(unsigned)grid, RT, 0, st>>>(
        records, vals, tile_ranges, vs, bg0, bg1, bg2, images, final_T, n_processed,
        &hdr->raster_tiles, &hdr->status, hdr->counters);
  return cudaGetLastError();
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
  if (g_bwd_occ == 0) {
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, raster_bwd_kernel<false>, RT, 0)) != cudaSuccess)
      return e;
    g_bwd_occ = occ > 0 ? occ : 1;
  }
  int64_t grid = (int64_t)sm_count() * g_bwd_occ;
  if (grid > vs.total_tiles) grid = vs.total_tiles;
  if (grid < 1) grid = 1;
  if (instrumented())
    raster_bwd_kernel<true><<<(unsigned)grid, RT, 0, st>>>(
        records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d,
        &hdr->backward_tiles, &hdr->status, hdr->counters);
  else
    raster_bwd_kernel<false><<<(unsigned)grid, RT, 0, st>>>(
        records, vals, tile_ranges, vs, bg0, bg1, bg2, final_T, n_processed, dL_dimages, g2d,
        &hdr->backward_tiles, &hdr->status, hdr->counters);
  return cudaGetLastError();
}

}  // namespace fgs
