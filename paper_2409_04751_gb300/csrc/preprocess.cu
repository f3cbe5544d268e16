// preprocess.cu - per-Gaussian preprocess (forward) and its backward, sm_103a.
//
// Forward (Sec. 4.1 preprocessCUDA with the fisheye projection of Sec. 4.2 / 4.3): one thread
// per Gaussian, looping over the views of the call, so each Gaussian's parameters (236 B at SH
// degree 3) are read from HBM once however many views there are (a later view finds its SH
// row in L1). Quaternions and SH rows are read with 16-byte vector loads when their rows are
// 16-byte aligned.
//
// Backward (Sec. 4.2 / 4.3 backward): one thread per Gaussian; the per-view screen-space
// gradients (written by the rasterizer backward) are pulled back through the conic,
// Sigma_p = T Sigma T^T, T = J W, J(mu_c) and the SH colour, summed over views, then through
// Sigma = R S S^T R^T to scales and quaternions.
#include "fgs_internal.cuh"

namespace fgs {

namespace {

template <bool VEC>
__device__ __forceinline__ float4 load_quat(const float *__restrict__ q, int64_t i) {
  if (VEC) return __ldg(reinterpret_cast<const float4 *>(q) + i);
  return make_float4(__ldg(q + 4 * i), __ldg(q + 4 * i + 1), __ldg(q + 4 * i + 2), __ldg(q + 4 * i + 3));
}

// Sigma = M M^T, M = R diag(s): upper triangle (xx, xy, xz, yy, yz, zz)
__device__ __forceinline__ void covariance(const float *R, float sx, float sy, float sz, float *S) {
  float M[9] = {R[0] * sx, R[1] * sy, R[2] * sz, R[3] * sx, R[4] * sy, R[5] * sz,
                R[6] * sx, R[7] * sy, R[8] * sz};
  S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

template <int D, bool VEC>
// five 256-thread CTAs per SM (at most 51 registers a thread, a few spilled to L1): more
// Gaussians in flight hide more of the parameter loads' latency than the spills cost
// (0.034 -> 0.031 ms on 500k Gaussians; six CTAs at 40 registers gain nothing)
__global__ void __launch_bounds__(256, 5)
    preprocess_fwd_kernel(GaussPtrs g, Views vs, fgs_record *__restrict__ rec,
                          uint32_t *__restrict__ tt) {
  constexpr int K = (D + 1) * (D + 1);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const float mx = __ldg(g.means + 3 * i), my = __ldg(g.means + 3 * i + 1),
              mz = __ldg(g.means + 3 * i + 2);
  const float op = __ldg(g.opacities + i);
  const bool op_ok = op >= ALPHA_MIN;

  // view-independent: Sigma and the footprint level q* = 2 ln(255 opacity)
  float S[6] = {0, 0, 0, 0, 0, 0};
  float qs = 0.f;
  // issued with the mean and opacity, not after the opacity test: one memory round trip
  const float4 q = load_quat<VEC>(g.quats, i);
  const float sx = __ldg(g.scales + 3 * i), sy = __ldg(g.scales + 3 * i + 1),
              sz = __ldg(g.scales + 3 * i + 2);
  if (op_ok) {
    float qn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float R[9];
    quat_to_rot(q.x * qn, q.y * qn, q.z * qn, q.w * qn, R);
    covariance(R, sx, sy, sz, S);
    qs = fmaxf(2.f * logf(255.f * op), 0.f);
  }

  for (int v = 0; v < vs.n; ++v) {
    const View &V = vs.v[v];
    const int64_t r = (int64_t)v * g.n + i;
    const float x = fmaf(V.W[0], mx, fmaf(V.W[1], my, fmaf(V.W[2], mz, V.b[0])));
    const float y = fmaf(V.W[3], mx, fmaf(V.W[4], my, fmaf(V.W[5], mz, V.b[1])));
    const float z = fmaf(V.W[6], mx, fmaf(V.W[7], my, fmaf(V.W[8], mz, V.b[2])));
    const float l2 = x * x + y * y + z * z;
    const float dist = sqrtf(l2);
    if (!(op_ok && dist > NEAR_DIST && in_field(V.model, x, y, z, dist))) {
      tt[r] = 0u;
      continue;
    }
    // mean (Sec. 3.2; other models Sec. 3.2 / Sec. 6) and Jacobian (Sec. 4.2)
    float px, py, J[6];
    project_mean(V, x, y, z, l2, px, py, J);
    if (V.model == FGS_CAM_PINHOLE && !in_pinhole_guard(V, px, py)) {
      tt[r] = 0u;
      continue;
    }
    const float J00 = J[0], J01 = J[1], J02 = J[2], J10 = J[3], J11 = J[4], J12 = J[5];
    // T = J W
    float T0[3], T1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T0[c] = J00 * V.W[c] + J01 * V.W[3 + c] + J02 * V.W[6 + c];
      T1[c] = J10 * V.W[c] + J11 * V.W[3 + c] + J12 * V.W[6 + c];
    }
    // Sigma_p = T Sigma T^T + 0.3 I (Sec. 4.3)
    const float u0 = T0[0] * S[0] + T0[1] * S[1] + T0[2] * S[2];
    const float u1 = T0[0] * S[1] + T0[1] * S[3] + T0[2] * S[4];
    const float u2 = T0[0] * S[2] + T0[1] * S[4] + T0[2] * S[5];
    const float w0 = T1[0] * S[0] + T1[1] * S[1] + T1[2] * S[2];
    const float w1 = T1[0] * S[1] + T1[1] * S[3] + T1[2] * S[4];
    const float w2 = T1[0] * S[2] + T1[1] * S[4] + T1[2] * S[5];
    const float a = u0 * T0[0] + u1 * T0[1] + u2 * T0[2] + DILATION;
    const float b = u0 * T1[0] + u1 * T1[1] + u2 * T1[2];
    const float c = w0 * T1[0] + w1 * T1[1] + w2 * T1[2] + DILATION;
    const float det = a * c - b * b;
    const float idet = 1.f / det;
    // footprint: AABB of the alpha >= 1/255 ellipse, padded, as an inclusive tile rect
    const float ex = fmaf(sqrtf(qs * a), 1.00001f, 1e-3f);
    const float ey = fmaf(sqrtf(qs * c), 1.00001f, 1e-3f);
    const float lx = (px - ex) * (1.f / TILE), hx = (px + ex) * (1.f / TILE);
    const float ly = (py - ey) * (1.f / TILE), hy = (py + ey) * (1.f / TILE);
    if (!(hx >= 0.f && hy >= 0.f && lx < (float)V.tiles_x && ly < (float)V.tiles_y)) {
      tt[r] = 0u;
      continue;
    }
    const int x0 = lx < 0.f ? 0 : (int)floorf(lx);
    const int y0 = ly < 0.f ? 0 : (int)floorf(ly);
    const int x1 = (int)floorf(fminf(hx, (float)(V.tiles_x - 1)));
    const int y1 = (int)floorf(fminf(hy, (float)(V.tiles_y - 1)));
    // colour from SH along (mu - camera centre); the coefficients are streamed in as they
    // are used (a later view of the call finds them in L1) rather than held in registers
    float dx = mx - V.cam_pos[0], dy = my - V.cam_pos[1], dz = mz - V.cam_pos[2];
    const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dn; dy *= dn; dz *= dn;
    float Y[K];
    sh_basis<D>(dx, dy, dz, Y);
    float rgb[3] = {0.5f, 0.5f, 0.5f};
    const float *shp = g.sh + (size_t)i * K * 3;
    if (VEC && ((K * 3) % 4) == 0) {
#pragma unroll
      for (int q = 0; q < K * 3 / 4; ++q) {
        const float4 w = __ldg(reinterpret_cast<const float4 *>(shp) + q);
        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int j = 4 * q + t;
          rgb[j % 3] = fmaf(wv[t], Y[j / 3], rgb[j % 3]);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < K * 3; ++j) rgb[j % 3] = fmaf(__ldg(shp + j), Y[j / 3], rgb[j % 3]);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaxf(rgb[ch], 0.f);
    float4 *o = reinterpret_cast<float4 *>(rec + r);
    o[0] = make_float4(px, py, c * idet, -b * idet);
    o[1] = make_float4(a * idet, op, rgb[0], rgb[1]);
    const uint32_t r01 = (uint32_t)x0 | ((uint32_t)y0 << 16);
    const uint32_t r23 = (uint32_t)x1 | ((uint32_t)y1 << 16);
    o[2] = make_float4(rgb[2], dist, __uint_as_float(r01), __uint_as_float(r23));
    tt[r] = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
  }
}

constexpr int PRE_BWD_THREADS = 128;

// The SH gradient rows of a block's Gaussians are accumulated in shared memory (one private
// row per thread, padded to an odd stride so that the threads' rows fall in distinct banks)
// and written out together at the end as one contiguous, coalesced block; the SH
// coefficients are read as they are needed. Neither is held in registers, which keeps enough
// warps resident to hide the memory latency.
template <int D, bool VEC>
// five CTAs per SM at 96 registers a thread (no spills): 0.063 -> 0.058 ms on 500k Gaussians
// against four at 128; six (80 registers, spilling) gain nothing
__global__ void __launch_bounds__(PRE_BWD_THREADS, 5)
    preprocess_bwd_kernel(GaussPtrs g, Views vs, const fgs_record *__restrict__ rec,
                          const uint32_t *__restrict__ tt, const float *__restrict__ g2d,
                          float *__restrict__ d_means, float *__restrict__ d_scales,
                          float *__restrict__ d_quats, float *__restrict__ d_opac,
                          float *__restrict__ d_sh) {
  constexpr int K = (D + 1) * (D + 1);
  constexpr int K3 = K * 3, KS = K3 + 1;
  __shared__ float s_dsh[PRE_BWD_THREADS * KS];
  float *my_dsh = s_dsh + threadIdx.x * KS;
  const int64_t i0 = (int64_t)blockIdx.x * PRE_BWD_THREADS;
  const int64_t i = i0 + threadIdx.x;
  const bool in = i < g.n;
  float dmu[3] = {0.f, 0.f, 0.f};
  float dS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma (symmetric, xx xy xz yy yz zz)
  float dop = 0.f;
  bool any = false;
  float S[6], R[9], qnv[4], qnorm = 1.f;
  const float mx = in ? __ldg(g.means + 3 * i) : 0.f, my = in ? __ldg(g.means + 3 * i + 1) : 0.f,
              mz = in ? __ldg(g.means + 3 * i + 2) : 0.f;
  const float *shp = g.sh + (size_t)(in ? i : 0) * K3;
  // issued with the mean, not after the visibility test: one memory round trip fewer
  const float4 q0 = in ? load_quat<VEC>(g.quats, i) : make_float4(1.f, 0.f, 0.f, 0.f);
  const float sc0 = in ? __ldg(g.scales + 3 * i) : 1.f, sc1 = in ? __ldg(g.scales + 3 * i + 1) : 1.f,
              sc2 = in ? __ldg(g.scales + 3 * i + 2) : 1.f;

  for (int v = 0; in && v < vs.n; ++v) {
    const int64_t r = (int64_t)v * g.n + i;
    if (tt[r] == 0u) continue;
    const View &V = vs.v[v];
    const bool first = !any;
    if (first) {
      any = true;
      const float4 q = q0;
      qnorm = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
      const float iq = 1.f / qnorm;
      qnv[0] = q.x * iq; qnv[1] = q.y * iq; qnv[2] = q.z * iq; qnv[3] = q.w * iq;
      quat_to_rot(qnv[0], qnv[1], qnv[2], qnv[3], R);
      covariance(R, sc0, sc1, sc2, S);
    }
    // the rasterizer backward leaves, per record, the moments of dL/dp over the pixel offsets
    // d = pixel - xy (p = -0.5 d^T conic d): m = sum dL/dp (dx, dy, dx^2, dx dy, dy^2), then
    // sum dL/dalpha alpha_raw and dL/drgb. With the record's conic (A, B, C) and opacity:
    //   dL/dxy = (A m_x + B m_y, B m_x + C m_y), dL/dA = -m_xx / 2, dL/dB = -m_xy,
    //   dL/dC = -m_yy / 2, dL/dopacity = sum dL/dalpha alpha_raw / opacity.
    const float4 m0 = __ldg(reinterpret_cast<const float4 *>(g2d + (size_t)r * G2D_STRIDE));
    const float4 m1 = __ldg(reinterpret_cast<const float4 *>(g2d + (size_t)r * G2D_STRIDE) + 1);
    const float gb = __ldg(g2d + (size_t)r * G2D_STRIDE + 8);
    const float4 rc0 = __ldg(reinterpret_cast<const float4 *>(rec + r));
    const float4 rc1 = __ldg(reinterpret_cast<const float4 *>(rec + r) + 1);
    const float rgb2 = __ldg(reinterpret_cast<const float *>(rec + r) + 8);
    const float4 g0 = make_float4(rc0.z * m0.x + rc0.w * m0.y, rc0.w * m0.x + rc1.x * m0.y,
                                  -0.5f * m0.z, -m0.w);
    const float4 g1 = make_float4(-0.5f * m1.x, m1.y / rc1.y, m1.z, m1.w);
    dop += g1.y;

    const float x = fmaf(V.W[0], mx, fmaf(V.W[1], my, fmaf(V.W[2], mz, V.b[0])));
    const float y = fmaf(V.W[3], mx, fmaf(V.W[4], my, fmaf(V.W[5], mz, V.b[1])));
    const float z = fmaf(V.W[6], mx, fmaf(V.W[7], my, fmaf(V.W[8], mz, V.b[2])));
    const float l2 = x * x + y * y + z * z;
    float pxm, pym, J[6];
    project_mean(V, x, y, z, l2, pxm, pym, J);
    (void)pxm;
    (void)pym;
    const float J00 = J[0], J01 = J[1], J02 = J[2], J10 = J[3], J11 = J[4], J12 = J[5];
    float T0[3], T1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T0[c] = J00 * V.W[c] + J01 * V.W[3 + c] + J02 * V.W[6 + c];
      T1[c] = J10 * V.W[c] + J11 * V.W[3 + c] + J12 * V.W[6 + c];
    }
    // conic -> Sigma_p: dL/dSigma_p = -M Gc M with M the conic matrix and Gc the symmetric
    // gradient [[gA, gB/2], [gB/2, gC]] (B is the off-diagonal entry, counted twice).
    const float cA = rc0.z, cB = rc0.w, cC = rc1.x;
    const float gA = g0.z, gBh = 0.5f * g0.w, gC = g1.x;
    const float t00 = gA * cA + gBh * cB, t01 = gA * cB + gBh * cC;
    const float t10 = gBh * cA + gC * cB, t11 = gBh * cB + gC * cC;
    const float Gs00 = -(cA * t00 + cB * t10);
    const float Gs01 = -(cA * t01 + cB * t11);
    const float Gs11 = -(cB * t01 + cC * t11);
    // dL/dSigma += T^T Gs T ; dL/dT = 2 Gs T Sigma
    float GsT0[3], GsT1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      GsT0[c] = Gs00 * T0[c] + Gs01 * T1[c];
      GsT1[c] = Gs01 * T0[c] + Gs11 * T1[c];
    }
    dS[0] += T0[0] * GsT0[0] + T1[0] * GsT1[0];
    dS[1] += T0[0] * GsT0[1] + T1[0] * GsT1[1];
    dS[2] += T0[0] * GsT0[2] + T1[0] * GsT1[2];
    dS[3] += T0[1] * GsT0[1] + T1[1] * GsT1[1];
    dS[4] += T0[1] * GsT0[2] + T1[1] * GsT1[2];
    dS[5] += T0[2] * GsT0[2] + T1[2] * GsT1[2];
    // GT = 2 (Gs T) Sigma
    float GT0[3], GT1[3];
    GT0[0] = 2.f * (GsT0[0] * S[0] + GsT0[1] * S[1] + GsT0[2] * S[2]);
    GT0[1] = 2.f * (GsT0[0] * S[1] + GsT0[1] * S[3] + GsT0[2] * S[4]);
    GT0[2] = 2.f * (GsT0[0] * S[2] + GsT0[1] * S[4] + GsT0[2] * S[5]);
    GT1[0] = 2.f * (GsT1[0] * S[0] + GsT1[1] * S[1] + GsT1[2] * S[2]);
    GT1[1] = 2.f * (GsT1[0] * S[1] + GsT1[1] * S[3] + GsT1[2] * S[4]);
    GT1[2] = 2.f * (GsT1[0] * S[2] + GsT1[1] * S[4] + GsT1[2] * S[5]);
    // dL/dJ = dL/dT W^T
    float GJ0[3], GJ1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      GJ0[k] = GT0[0] * V.W[3 * k] + GT0[1] * V.W[3 * k + 1] + GT0[2] * V.W[3 * k + 2];
      GJ1[k] = GT1[0] * V.W[3 * k] + GT1[1] * V.W[3 * k + 1] + GT1[2] * V.W[3 * k + 2];
    }
    // J -> mu_c (Sec. 4.3 for the equidistant model; the other models alike)
    const float GJ[6] = {GJ0[0], GJ0[1], GJ0[2], GJ1[0], GJ1[1], GJ1[2]};
    float dmc0, dmc1, dmc2;
    jacobian_backward(V, x, y, z, l2, GJ, dmc0, dmc1, dmc2);
    // mu_p -> mu_c (Sec. 4.2): J^T dL/dmu_p
    dmc0 += J00 * g0.x + J10 * g0.y;
    dmc1 += J01 * g0.x + J11 * g0.y;
    dmc2 += J02 * g0.x + J12 * g0.y;
    // mu_c = W mu + b
    dmu[0] += V.W[0] * dmc0 + V.W[3] * dmc1 + V.W[6] * dmc2;
    dmu[1] += V.W[1] * dmc0 + V.W[4] * dmc1 + V.W[7] * dmc2;
    dmu[2] += V.W[2] * dmc0 + V.W[5] * dmc1 + V.W[8] * dmc2;
    // colour -> SH and view direction (clamped channels pass no gradient)
    const float grgb[3] = {rc1.z > 0.f ? g1.z : 0.f, rc1.w > 0.f ? g1.w : 0.f,
                           rgb2 > 0.f ? gb : 0.f};
    float ux = mx - V.cam_pos[0], uy = my - V.cam_pos[1], uz = mz - V.cam_pos[2];
    const float un = rsqrtf(ux * ux + uy * uy + uz * uz);
    ux *= un; uy *= un; uz *= un;
    float Y[K], dY[K][3];
    sh_basis<D>(ux, uy, uz, Y);
    sh_basis_grad<D>(ux, uy, uz, dY);
    // s_k = <SH row k, dL/drgb>, each over the channels in order 0, 1, 2; the coefficients
    // come in as 16-byte loads where the rows allow it (the same sums either way)
    float sk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) sk[k] = 0.f;
    if (VEC && (K3 % 4) == 0) {
#pragma unroll
      for (int q = 0; q < K3 / 4; ++q) {
        const float4 w = __ldg(reinterpret_cast<const float4 *>(shp) + q);
        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int j = 4 * q + t;
          sk[j / 3] = fmaf(wv[t], grgb[j % 3], sk[j / 3]);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < K3; ++j) sk[j / 3] = fmaf(__ldg(shp + j), grgb[j % 3], sk[j / 3]);
    }
    float dd0 = 0.f, dd1 = 0.f, dd2 = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const int j = 3 * k + ch;
        my_dsh[j] = fmaf(Y[k], grgb[ch], first ? 0.f : my_dsh[j]);
      }
      dd0 = fmaf(sk[k], dY[k][0], dd0);
      dd1 = fmaf(sk[k], dY[k][1], dd1);
      dd2 = fmaf(sk[k], dY[k][2], dd2);
    }
    const float dot = ux * dd0 + uy * dd1 + uz * dd2;
    dmu[0] += (dd0 - ux * dot) * un;
    dmu[1] += (dd1 - uy * dot) * un;
    dmu[2] += (dd2 - uz * dot) * un;
  }

  float dsc[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
  if (any) {
    // Sigma = M M^T, M = R diag(s): dL/dM = 2 dS M
    const float sx = __ldg(g.scales + 3 * i), sy = __ldg(g.scales + 3 * i + 1),
                sz = __ldg(g.scales + 3 * i + 2);
    const float sc[3] = {sx, sy, sz};
    const float dSf[9] = {dS[0], dS[1], dS[2], dS[1], dS[3], dS[4], dS[2], dS[4], dS[5]};
    float GR[9];
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        // (dS M)[rr][cc] = sum_k dS[rr][k] R[k][cc] s_cc
        const float gm = 2.f * (dSf[3 * rr] * R[cc] + dSf[3 * rr + 1] * R[3 + cc] +
                                dSf[3 * rr + 2] * R[6 + cc]) * sc[cc];
        dsc[cc] += gm * R[3 * rr + cc];
        GR[3 * rr + cc] = gm * sc[cc];
      }
    const float w = qnv[0], x = qnv[1], y = qnv[2], z = qnv[3];
    // dL/dq_n from R(q_n), entry by entry
    const float gw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    const float gx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] +
                            z * GR[6] + w * GR[7] - 2.f * x * GR[8]);
    const float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] -
                            w * GR[6] + z * GR[7] - 2.f * y * GR[8]);
    const float gz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] +
                            y * GR[5] + x * GR[6] + y * GR[7]);
    // through q_n = q / |q|
    const float dot = gw * w + gx * x + gy * y + gz * z;
    const float iq = 1.f / qnorm;
    dq[0] = (gw - w * dot) * iq; dq[1] = (gx - x * dot) * iq;
    dq[2] = (gy - y * dot) * iq; dq[3] = (gz - z * dot) * iq;
  }
  if (in) {
    d_means[3 * i] = dmu[0]; d_means[3 * i + 1] = dmu[1]; d_means[3 * i + 2] = dmu[2];
    d_scales[3 * i] = dsc[0]; d_scales[3 * i + 1] = dsc[1]; d_scales[3 * i + 2] = dsc[2];
    d_quats[4 * i] = dq[0]; d_quats[4 * i + 1] = dq[1]; d_quats[4 * i + 2] = dq[2]; d_quats[4 * i + 3] = dq[3];
    d_opac[i] = dop;
    if (!any) {
#pragma unroll
      for (int j = 0; j < K3; ++j) my_dsh[j] = 0.f;
    }
  }
  __syncthreads();
  // the block's rows are contiguous in d_sh: consecutive threads store consecutive floats
  const int64_t rows = g.n - i0 < PRE_BWD_THREADS ? g.n - i0 : PRE_BWD_THREADS;
  float *dst = d_sh + (size_t)i0 * K3;
  for (int j = threadIdx.x; j < rows * K3; j += PRE_BWD_THREADS)
    dst[j] = s_dsh[(j / K3) * KS + j % K3];
}

template <int D>
cudaError_t fwd_dispatch(const GaussPtrs &g, const Views &vs, fgs_record *rec, uint32_t *tt,
                         bool vec, cudaStream_t st) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((g.n + threads - 1) / threads);
  if (vec) preprocess_fwd_kernel<D, true><<<blocks, threads, 0, st>>>(g, vs, rec, tt);
  else preprocess_fwd_kernel<D, false><<<blocks, threads, 0, st>>>(g, vs, rec, tt);
  return cudaGetLastError();
}

template <int D>
cudaError_t bwd_dispatch(const GaussPtrs &g, const Views &vs, const fgs_record *rec,
                         const uint32_t *tt, const float *g2d, float *dm, float *ds, float *dq,
                         float *dop, float *dsh, bool vec, cudaStream_t st) {
  const int threads = PRE_BWD_THREADS;
  const unsigned blocks = (unsigned)((g.n + threads - 1) / threads);
  if (vec)
    preprocess_bwd_kernel<D, true><<<blocks, threads, 0, st>>>(g, vs, rec, tt, g2d, dm, ds, dq, dop, dsh);
  else
    preprocess_bwd_kernel<D, false><<<blocks, threads, 0, st>>>(g, vs, rec, tt, g2d, dm, ds, dq, dop, dsh);
  return cudaGetLastError();
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cudaError_t launch_preprocess_fwd(const GaussPtrs &g, const Views &vs, fgs_record *records,
                                  uint32_t *tiles_touched, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  const bool vec = aligned16(g.quats) && aligned16(g.sh);
  switch (g.sh_degree) {
    case 0: return fwd_dispatch<0>(g, vs, records, tiles_touched, vec, st);
    case 1: return fwd_dispatch<1>(g, vs, records, tiles_touched, vec, st);
    case 2: return fwd_dispatch<2>(g, vs, records, tiles_touched, vec, st);
    default: return fwd_dispatch<3>(g, vs, records, tiles_touched, vec, st);
  }
}

cudaError_t launch_preprocess_bwd(const GaussPtrs &g, const Views &vs, const fgs_record *records,
                                  const uint32_t *tiles_touched, const float *g2d,
                                  float *d_means, float *d_scales, float *d_quats,
                                  float *d_opacities, float *d_sh, uint32_t *status,
                                  cudaStream_t st) {
  (void)status;
  if (g.n == 0) return cudaSuccess;
  const bool vec = aligned16(g.quats) && aligned16(g.sh) && aligned16(d_sh);
  switch (g.sh_degree) {
    case 0: return bwd_dispatch<0>(g, vs, records, tiles_touched, g2d, d_means, d_scales, d_quats, d_opacities, d_sh, vec, st);
    case 1: return bwd_dispatch<1>(g, vs, records, tiles_touched, g2d, d_means, d_scales, d_quats, d_opacities, d_sh, vec, st);
    case 2: return bwd_dispatch<2>(g, vs, records, tiles_touched, g2d, d_means, d_scales, d_quats, d_opacities, d_sh, vec, st);
    default: return bwd_dispatch<3>(g, vs, records, tiles_touched, g2d, d_means, d_scales, d_quats, d_opacities, d_sh, vec, st);
  }
}

}  // namespace fgs
