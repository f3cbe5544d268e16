// train.cu - the optimisation loop around the rendering path (Sec. 5.1 "Optimization": the
// models are trained with the loss, optimiser and hyperparameters of the renderer the method
// plugs into, i.e. Adam on per-Gaussian parameters), sm_103a.
//
//  loss_l1_kernel   L = scale * sum |image - target| and dL/dimage = scale * sign(image - target)
//                   (0 where equal), one grid-stride pass, the sum by warp shuffles and one
//                   atomic per warp.
//  adam_kernel      one launch over several parameter tensors ("groups"), after a one-thread
//                   launch that advances the device step counter (so a captured graph replays
//                   with the right bias correction): for each element the
//                   gradient of the raw parameter from that of its activated value
//                   (identity, exp, sigmoid), Adam's moment updates with bias correction
//                   (Kingma & Ba, Algorithm 1), the raw update, and the activated value written
//                   for the next render. CTAs are assigned to groups by a block prefix.
#include "fgs_internal.cuh"

namespace fgs {
namespace {

__global__ void __launch_bounds__(256)
    loss_l1_kernel(const float *__restrict__ image, const float *__restrict__ target,
                   float *__restrict__ grad, int64_t n, float scale, float *loss) {
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = image[i] - target[i];
    acc += fabsf(d);
    grad[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.f) atomicAdd(loss, acc * scale);
}

struct AdamArgs {
  fgs_adam_group g[FGS_ADAM_MAX_GROUPS];
  int64_t block_start[FGS_ADAM_MAX_GROUPS + 1];
  int n_groups;
  double beta1d, beta2d;  // for the bias corrections 1 / (1 - beta^t)
  float beta1, beta2, eps;
  float omb1, omb2;       // 1 - beta1, 1 - beta2, rounded once from double
  const int64_t *step;    // the step number t (>= 1), read on the device
};

constexpr int ADAM_THREADS = 256;
constexpr int ADAM_ITEMS = 4;

// the step counter: t <- t + 1 before the update that uses it
__global__ void count_step_kernel(int64_t *step) { *step += 1; }

__global__ void __launch_bounds__(ADAM_THREADS) adam_kernel(AdamArgs a) {
  __shared__ float s_c[2];  // 1 / (1 - beta1^t), 1 / (1 - beta2^t)
  if (threadIdx.x == 0) {
    const double t = (double)*a.step;
    s_c[0] = (float)(1.0 / (1.0 - pow(a.beta1d, t)));
    s_c[1] = (float)(1.0 / (1.0 - pow(a.beta2d, t)));
  }
  __syncthreads();
  const float c1 = s_c[0], c2 = s_c[1];
  int k = 0;
  while (k + 1 < a.n_groups && (int64_t)blockIdx.x >= a.block_start[k + 1]) ++k;
  const fgs_adam_group &G = a.g[k];
  const int64_t base = ((int64_t)blockIdx.x - a.block_start[k]) * ADAM_THREADS * ADAM_ITEMS;
#pragma unroll
  for (int it = 0; it < ADAM_ITEMS; ++it) {
    const int64_t i = base + it * ADAM_THREADS + threadIdx.x;
    if (i >= G.count) break;
    const float raw = G.raw[i];
    float gr = G.grad[i];
    // d act / d raw at the current raw value (the one the gradient was taken at)
    if (G.activation == FGS_ACT_EXP) {
      gr *= expf(raw);
    } else if (G.activation == FGS_ACT_SIGMOID) {
      const float s = 1.f / (1.f + expf(-raw));
      gr *= s * (1.f - s);
    }
    const float m = fmaf(a.beta1, G.m[i], a.omb1 * gr);
    const float v = fmaf(a.beta2, G.v[i], a.omb2 * gr * gr);
    G.m[i] = m;
    G.v[i] = v;
    const float upd = G.lr * (m * c1) / (sqrtf(v * c2) + a.eps);
    const float nr = raw - upd;
    G.raw[i] = nr;
    if (G.act != nullptr && G.act != G.raw) {
      float act = nr;
      if (G.activation == FGS_ACT_EXP) act = expf(nr);
      else if (G.activation == FGS_ACT_SIGMOID) act = 1.f / (1.f + expf(-nr));
      G.act[i] = act;
    }
  }
}

}  // namespace
}  // namespace fgs

using namespace fgs;

extern "C" {

fgs_status fgs_loss_l1(const float *images, const float *targets, float *dL_dimages, int64_t n,
                       float scale, float *loss, fgs_stream stream) {
  if (n < 0 || !images || !targets || !dL_dimages || !loss || !(scale >= 0.f))
    return FGS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return FGS_ERR_CUDA;
  if (n == 0) return FGS_OK;
  int64_t grid = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  if (grid > cap) grid = cap;
  loss_l1_kernel<<<(unsigned)grid, 256, 0, st>>>(images, targets, dL_dimages, n, scale, loss);
  return cudaGetLastError() == cudaSuccess ? FGS_OK : FGS_ERR_CUDA;
}

fgs_status fgs_adam_step(const fgs_adam_group *groups, int n_groups, double beta1,
                         double beta2, float eps, int64_t *step, fgs_stream stream) {
  if (!groups || n_groups < 1 || n_groups > FGS_ADAM_MAX_GROUPS || !step) return FGS_ERR_INVALID_ARG;
  if (!(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps > 0.f))
    return FGS_ERR_INVALID_ARG;
  AdamArgs a;
  memset(&a, 0, sizeof a);
  a.n_groups = n_groups;
  a.beta1d = beta1;
  a.beta2d = beta2;
  a.beta1 = (float)beta1;
  a.beta2 = (float)beta2;
  a.eps = eps;
  a.omb1 = (float)(1.0 - beta1);
  a.omb2 = (float)(1.0 - beta2);
  a.step = step;
  int64_t blocks = 0;
  for (int k = 0; k < n_groups; ++k) {
    const fgs_adam_group &G = groups[k];
    if (G.count < 0 || G.activation < FGS_ACT_NONE || G.activation > FGS_ACT_SIGMOID)
      return FGS_ERR_INVALID_ARG;
    if (G.count > 0 && (!G.raw || !G.grad || !G.m || !G.v)) return FGS_ERR_INVALID_ARG;
    a.g[k] = G;
    a.block_start[k] = blocks;
    blocks += (G.count + ADAM_THREADS * ADAM_ITEMS - 1) / (ADAM_THREADS * ADAM_ITEMS);
  }
  a.block_start[n_groups] = blocks;
  if (blocks > 0x7fffffffLL) return FGS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  count_step_kernel<<<1, 1, 0, st>>>(step);
  if (blocks > 0) adam_kernel<<<(unsigned)blocks, ADAM_THREADS, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? FGS_OK : FGS_ERR_CUDA;
}

}  // extern "C"
