// S8: Adam (Kingma & Ba) with I-NGP's settings, one optimiser per tile (its
// hash table and density MLP) and one per colour MLP, none of them reset when
// the window moves (Sec. 4.1, 4.4, 4.6).  The update is fused with zeroing
// the gradient accumulator and, for mixed precision, with refreshing the
// FP16 working copy of tables and weights and with the loss-scale logic:
// a step whose gradients are not all finite is skipped, the scale halved.
#include "kernels.cuh"

namespace snk {
namespace {

__global__ void k_check_finite(const float *__restrict__ g, int64_t n, snk_state *state) {
  bool bad = false;
  const int64_t n4 = n / 4;
  const float4 *g4 = reinterpret_cast<const float4 *>(g);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = g4[i];
    bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
  }
  for (int64_t i = n4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(g[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&state->reserved[0], 1u);
}

__global__ void k_adam(const AdamArgs a) {
  const bool skip = a.mixed && a.state->reserved[0] != 0u;
  const float inv_scale = a.mixed ? 1.0f / a.state->loss_scale : 1.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    int g = 0;
    for (int k = 0; k < a.n_groups; ++k)
      if (i >= a.start[k] && i < a.end[k]) g = k;
    const float grad = a.grads[i];
    a.grads[i] = 0.0f;
    if (skip) continue;
    const bool mlp = i >= a.mlp_start[g];
    float w = a.params[i];
    float gr = grad * inv_scale;
    if (mlp) gr = fmaf(a.l2, w, gr);
    const float t = (float)(a.steps[g] + 1);
    float m = a.m[i], v = a.v[i];
    m = fmaf(a.beta1, m, (1.0f - a.beta1) * gr);
    v = fmaf(a.beta2, v, (1.0f - a.beta2) * gr * gr);
    const float bc1 = 1.0f - powf(a.beta1, t), bc2 = 1.0f - powf(a.beta2, t);
    w -= a.lr * (m / bc1) / (sqrtf(v / bc2) + a.eps);
    a.params[i] = w;
    a.m[i] = m;
    a.v[i] = v;
    if (a.params_lp) a.params_lp[i] = __half_as_ushort(__float2half_rn(w));
  }
}

// Bookkeeping after the update: step counts, loss scale, iteration counter.
__global__ void k_step_end(snk_state *state, int32_t *steps, int n_groups, int mixed) {
  const bool skip = mixed && state->reserved[0] != 0u;
  if (skip) {
    state->status |= kStatusOverflow;
    state->loss_scale = fmaxf(state->loss_scale * 0.5f, 1.0f);
    state->good_steps = 0;
  } else {
    for (int k = 0; k < n_groups; ++k) steps[k] += 1;
    if (mixed) {
      state->good_steps += 1;
      if (state->good_steps >= 2000) {
        state->loss_scale = fminf(state->loss_scale * 2.0f, 16777216.0f);
        state->good_steps = 0;
      }
    }
  }
  state->iteration += 1u;
}

}  // namespace

cudaError_t launch_adam(const AdamArgs &a, int sm_count, cudaStream_t st) {
  const int grid = sm_count * 8;
  if (a.mixed) k_check_finite<<<grid, 256, 0, st>>>(a.grads, a.n, a.state);
  k_adam<<<grid, 256, 0, st>>>(a);
  k_step_end<<<1, 1, 0, st>>>(a.state, a.steps, a.n_groups, a.mixed);
  count_launches(a.mixed ? 3 : 2);
  return cudaGetLastError();
}

}  // namespace snk
