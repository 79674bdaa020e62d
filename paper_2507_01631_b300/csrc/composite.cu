// S5 + S6 + S7a: front-to-back volume rendering of each ray over the samples
// of all its segments (NeRF Eq. 3, unchanged by the segmented sampler,
// Sec. 4.5), the colour loss against the target crop (Sec. 4.4, MSE over
// accepted rays) and the backward of the rendering.
//
// One warp per ray.  Forward: per 32-sample chunk a warp inclusive scan of
// tau = sigma * delta gives T_i = exp(-sum_{j<i} tau_j); alpha_i = 1 -
// exp(-tau_i) (computed as -expm1 so that thin samples keep their weight);
// w_i = T_i alpha_i.  The weights are kept in shared memory for the backward
// (rays of up to kParkChunks x 32 samples; longer ones park them in the
// gradient buffer).
// Backward (reverse chunk order, reverse warp scans): with g = dLoss/dC,
//   dLoss/dc_i     = w_i g
//   dLoss/dsigma_i = delta_i (T_{i+1} (g . c_i) - sum_{j>i} w_j (g . c_j)),
// where T_{i+1} = T_final + sum_{j>i} w_j is formed from positive suffix sums
// (no cancellation against the total).
#include "kernels.cuh"

namespace snk {
namespace {

__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// sum over lanes >= lane
__device__ __forceinline__ float warp_rev_scan(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v += t;
  }
  return v;
}

constexpr int kParkChunks = 16;  // 32-sample chunks of a ray whose weights stay in shared memory

__global__ void __launch_bounds__(512) k_composite(const CompositeArgs a) {
  extern __shared__ float wpark[];  // [warps of the block][kParkChunks][32]
  const int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  float *wp = wpark + (threadIdx.x >> 5) * kParkChunks * 32;
  if (r >= a.B) return;
  const bool none = a.state != nullptr && a.state->n_samples == 0u;
  uint32_t n[3], off[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    n[s] = none ? 0u : a.seg_n[(size_t)r * 3 + s];
    off[s] = a.seg_off[(size_t)r * 3 + s];
  }
  const float4 *sr = reinterpret_cast<const float4 *>(a.sigma_rgb);
  float4 *dsr = reinterpret_cast<float4 *>(a.dsr);
  // first chunk of each segment in the ray's chunk sequence; park in shared memory if all fit
  const int cs1 = (int)((n[0] + 31) / 32), cs2 = cs1 + (int)((n[1] + 31) / 32);
  const bool park = cs2 + (int)((n[2] + 31) / 32) <= kParkChunks;
  int chunk = 0;

  float carry = 0.f, cr = 0.f, cg = 0.f, cb = 0.f, dep = 0.f, op = 0.f;
#pragma unroll 1
  for (int s = 0; s < 3; ++s) {
    for (uint32_t base = 0; base < n[s]; base += 32) {
      const uint32_t i = base + lane;
      const bool v = i < n[s];
      const size_t q = (size_t)off[s] + i;
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      float t = 0.f, dt = 0.f;
      if (v) {
        c = sr[q];
        t = a.smp_t[q];
        dt = a.smp_dt[q];
      }
      const float tau = c.x * dt;
      const float incl = warp_incl_scan(tau, lane);
      const float T = expf(-(carry + (incl - tau)));
      const float w = T * -expm1f(-tau);
      cr = fmaf(w, c.y, cr);
      cg = fmaf(w, c.z, cg);
      cb = fmaf(w, c.w, cb);
      dep = fmaf(w, t, dep);
      op += w;
      if (dsr != nullptr) {
        if (park)
          wp[chunk * 32 + lane] = w;
        else if (v)
          dsr[q] = make_float4(w, 0.f, 0.f, 0.f);
      }
      ++chunk;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  cr = warp_sum(cr);
  cg = warp_sum(cg);
  cb = warp_sum(cb);
  dep = warp_sum(dep);
  op = warp_sum(op);
  const float t_final = expf(-carry);
  if (lane == 0) {
    if (a.out) {
      float *o = a.out + (size_t)r * 5;
      o[0] = cr;
      o[1] = cg;
      o[2] = cb;
      o[3] = dep;
      o[4] = op;
    }
    if (a.t_final) a.t_final[r] = t_final;
  }
  if (dsr == nullptr) return;
  const bool has = n[0] + n[1] + n[2] > 0;
  if (!has) return;

  float g0, g1, g2;
  if (a.train) {
    const uint32_t p = a.pix[r];
    const int v = (int)(p >> 24), row = (int)((p >> 12) & 0xFFFu), col = (int)(p & 0xFFFu);
    const DevView &cv = a.views[v];
    const float *gt = cv.crop + ((size_t)(row - cv.crop_r0) * cv.crop_w + (col - cv.crop_c0)) * 3;
    const float d0 = cr - gt[0], d1 = cg - gt[1], d2 = cb - gt[2];
    const float inv = 1.0f / (3.0f * (float)a.state->n_accepted);
    if (lane == 0) atomicAdd(&a.state->loss, (d0 * d0 + d1 * d1 + d2 * d2) * inv);
    const float k = 2.0f * inv * a.state->loss_scale;
    g0 = k * d0;
    g1 = k * d1;
    g2 = k * d2;
  } else {
    g0 = a.g_rgb[(size_t)r * 3 + 0];
    g1 = a.g_rgb[(size_t)r * 3 + 1];
    g2 = a.g_rgb[(size_t)r * 3 + 2];
  }

  float suf_w = 0.f, suf_wgc = 0.f;
#pragma unroll 1
  for (int s = 2; s >= 0; --s) {
    if (n[s] == 0) continue;
    const int nch = (int)((n[s] + 31) / 32);
    const int cs = s == 0 ? 0 : (s == 1 ? cs1 : cs2);
    for (int ch = nch - 1; ch >= 0; --ch) {
      const uint32_t i = (uint32_t)ch * 32 + lane;
      const bool v = i < n[s];
      const size_t q = (size_t)off[s] + i;
      float w = 0.f, dt = 0.f;
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      if (v) {
        w = park ? wp[(cs + ch) * 32 + lane] : dsr[q].x;
        c = sr[q];
        dt = a.smp_dt[q];
      }
      const float gc = g0 * c.y + g1 * c.z + g2 * c.w;
      const float wgc = w * gc;
      const float rw = warp_rev_scan(w, lane);
      const float rwgc = warp_rev_scan(wgc, lane);
      const float after_w = suf_w + (rw - w);
      const float after_wgc = suf_wgc + (rwgc - wgc);
      const float t_next = t_final + after_w;
      if (v) dsr[q] = make_float4(dt * (t_next * gc - after_wgc), w * g0, w * g1, w * g2);
      suf_w += __shfl_sync(0xffffffffu, rw, 0);
      suf_wgc += __shfl_sync(0xffffffffu, rwgc, 0);
    }
  }
}

}  // namespace

cudaError_t launch_composite(const CompositeArgs &a, cudaStream_t st, const Tuning &tu) {
  if (a.B <= 0) return cudaSuccess;
  const int64_t threads = (int64_t)a.B * 32;
  const int nt = tu.composite_threads;
  k_composite<<<(unsigned)((threads + nt - 1) / nt), nt, sizeof(float) * (nt / 32) * kParkChunks * 32, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace snk
