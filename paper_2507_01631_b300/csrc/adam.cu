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
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&state->nonfinite, 1u);
}

// Per optimiser group: the bias corrections 1 - beta^t of its step t = steps + 1.
__device__ __forceinline__ void bias_corrections(const AdamArgs &a, float *bc1, float *bc2) {
  if (threadIdx.x < a.n_groups) {
    const float t = (float)(a.steps[threadIdx.x] + 1);
    bc1[threadIdx.x] = 1.0f - powf(a.beta1, t);
    bc2[threadIdx.x] = 1.0f - powf(a.beta2, t);
  }
  __syncthreads();
}

__device__ __forceinline__ int group_of(const AdamArgs &a, int64_t i) {
  int g = 0;
  for (int k = 0; k < a.n_groups; ++k)
    if (i >= a.start[k] && i < a.end[k]) g = k;
  return g;
}

// One parameter: m, v, weight (I-NGP Adam with L2 on MLP weights); returns the new weight.
__device__ __forceinline__ float adam_one(const AdamArgs &a, float grad, float inv_scale, bool mlp, float bc1, float bc2,
                                          float &w, float &m, float &v) {
  float gr = grad * inv_scale;
  if (mlp) gr = fmaf(a.l2, w, gr);
  m = fmaf(a.beta1, m, (1.0f - a.beta1) * gr);
  v = fmaf(a.beta2, v, (1.0f - a.beta2) * gr * gr);
  w -= a.lr * (m / bc1) / (sqrtf(v / bc2) + a.eps);
  return w;
}

__global__ void k_adam(const AdamArgs a) {
  __shared__ float bc1[9], bc2[9];
  bias_corrections(a, bc1, bc2);
  const bool skip = a.mixed && a.state->nonfinite != 0u;
  const float inv_scale = a.mixed ? 1.0f / a.state->loss_scale : 1.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int g = group_of(a, i);
    const float grad = a.grads[i];
    a.grads[i] = 0.0f;
    if (skip) continue;
    float w = a.params[i], m = a.m[i], v = a.v[i];
    adam_one(a, grad, inv_scale, i >= a.mlp_start[g], bc1[g], bc2[g], w, m, v);
    a.params[i] = w;
    a.m[i] = m;
    a.v[i] = v;
    if (a.params_lp) a.params_lp[i] = __half_as_ushort(__float2half_rn(w));
  }
}

// The same update four parameters at a time (16-byte accesses); every group boundary and
// L2 boundary is a multiple of 4, so the four share a group and an L2 flag.  Each thread takes
// two such groups a round and issues all eight loads before using any (the skip test is uniform
// and rare, so the parameters are read even when it holds): more bytes in flight per thread.
__global__ void __launch_bounds__(256, 4) k_adam4(const AdamArgs a) {
  __shared__ float bc1[9], bc2[9];
  bias_corrections(a, bc1, bc2);
  const bool skip = a.mixed && a.state->nonfinite != 0u;
  const float inv_scale = a.mixed ? 1.0f / a.state->loss_scale : 1.0f;
  const int64_t n4 = a.n / 4;
  float4 *P = reinterpret_cast<float4 *>(a.params), *G = reinterpret_cast<float4 *>(a.grads);
  float4 *M = reinterpret_cast<float4 *>(a.m), *V = reinterpret_cast<float4 *>(a.v);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto update = [&](int64_t q, const float4 &gr, float4 &w, float4 &m, float4 &v) {
    const int64_t i = 4 * q;
    const int g = group_of(a, i);
    const bool mlp = i >= a.mlp_start[g];
    const float b1 = bc1[g], b2 = bc2[g];
    adam_one(a, gr.x, inv_scale, mlp, b1, b2, w.x, m.x, v.x);
    adam_one(a, gr.y, inv_scale, mlp, b1, b2, w.y, m.y, v.y);
    adam_one(a, gr.z, inv_scale, mlp, b1, b2, w.z, m.z, v.z);
    adam_one(a, gr.w, inv_scale, mlp, b1, b2, w.w, m.w, v.w);
    P[q] = w;
    M[q] = m;
    V[q] = v;
    if (a.params_lp) {
      const __half2 lo = __floats2half2_rn(w.x, w.y), hi = __floats2half2_rn(w.z, w.w);
      reinterpret_cast<uint2 *>(a.params_lp)[q] =
          make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
    }
  };
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t q0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q0 < n4; q0 += 2 * stride) {
    const int64_t q1 = q0 + stride;
    const bool two = q1 < n4;
    float4 g0 = G[q0], w0 = P[q0], m0 = M[q0], v0 = V[q0];
    float4 g1 = zero, w1 = zero, m1 = zero, v1 = zero;
    if (two) {
      g1 = G[q1];
      w1 = P[q1];
      m1 = M[q1];
      v1 = V[q1];
    }
    G[q0] = zero;
    if (two) G[q1] = zero;
    if (skip) continue;
    update(q0, g0, w0, m0, v0);
    if (two) update(q1, g1, w1, m1, v1);
  }
}

// Bookkeeping after the update: step counts, loss scale, iteration counter, the backward mode.
__global__ void k_step_end(snk_state *state, int32_t *steps, int n_groups, int mixed, uint32_t bwd_mode) {
  state->bwd_mode = bwd_mode;
  const bool skip = mixed && state->nonfinite != 0u;
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

// The FP16 working copy of binary32 parameters, round to nearest even (the conversion the Adam
// kernels apply after each update).
__global__ void k_refresh_lp(const float *__restrict__ w, uint16_t *__restrict__ lp, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    lp[i] = __half_as_ushort(__float2half_rn(w[i]));
}

}  // namespace

// Persistent grid-stride kernels: one wave of resident blocks (a second, partial wave would
// leave most SMs idle at its end).
template <typename K>
int blocks_per_sm(K kernel, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm;
}

cudaError_t launch_adam(const AdamArgs &a, int sm_count, cudaStream_t st) {
  static const int b_check = blocks_per_sm(k_check_finite, 256), b_adam = blocks_per_sm(k_adam, 256),
                   b_adam4 = blocks_per_sm(k_adam4, 256);
  const int g_check = sm_count * b_check, g_adam = sm_count * b_adam, g_adam4 = sm_count * b_adam4;
  if (a.mixed) k_check_finite<<<g_check, 256, 0, st>>>(a.grads, a.n, a.state);
  bool vec4 = a.n % 4 == 0 && a.n_groups <= 9;
  for (int k = 0; k < a.n_groups; ++k)
    vec4 = vec4 && a.start[k] % 4 == 0 && a.end[k] % 4 == 0 && a.mlp_start[k] % 4 == 0;
  auto aligned = [](const void *p, uintptr_t b) { return p == nullptr || reinterpret_cast<uintptr_t>(p) % b == 0; };
  vec4 = vec4 && aligned(a.params, 16) && aligned(a.grads, 16) && aligned(a.m, 16) && aligned(a.v, 16) &&
         aligned(a.params_lp, 8);
  if (vec4)
    k_adam4<<<g_adam4, 256, 0, st>>>(a);
  else
    k_adam<<<g_adam, 256, 0, st>>>(a);
  k_step_end<<<1, 1, 0, st>>>(a.state, a.steps, a.n_groups, a.mixed, a.bwd_mode);
  count_launches(a.mixed ? 3 : 2);
  return cudaGetLastError();
}

cudaError_t launch_refresh_lp(const float *w, uint16_t *lp, int64_t n, int sm_count, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_refresh_lp<<<sm_count * 8, 256, 0, st>>>(w, lp, n);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace snk
