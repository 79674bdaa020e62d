// S3 + S4 (+ S7b, S7c): the binary32 field path -- multiresolution hash
// encoding (Sec. 4.1, NGP) of each sample with its tile's table, the tile's
// density MLP, the colour MLP (shared across tiles, Sec. 4.1), and the fused
// backward that recomputes the forward activations instead of storing them,
// back-propagates through both MLPs, accumulates the weight gradients and
// scatter-adds the feature gradients into the hash tables.
//
// Work unit: a tile of 64 consecutive slot-major samples (always inside one
// parameter slot, because slot ranges start on multiples of 128).  128
// threads per block, two per sample; every layer is computed from rows held
// in shared memory.  Weight gradients live in registers (each thread owns a
// fixed set of weights) for the whole persistent loop and are flushed with
// one atomic per weight when the block moves to another slot and at exit.
//
// View-direction variant (VD): the colour MLP's input row is [g | SH_16(d)],
// the 16 real spherical harmonics of the sample's ray direction written next
// to g in the same shared-memory row; the input gradient of that layer is
// taken over the g columns only.
#include "kernels.cuh"

namespace snk {
namespace {

constexpr int NS = 64;   // samples per tile
constexpr int NT = 128;  // threads per block

template <int IN, int G, bool COL, bool VD>
struct Dims {
  static constexpr int H = kHidden;
  static constexpr int CIN = G + (VD ? 16 : 0);  // colour input width
  static constexpr int S0 = IN + 1, SH = H + 1, SG = CIN + 1;
  static constexpr int X0 = 0;
  static constexpr int X1 = X0 + NS * S0;
  static constexpr int X2 = X1 + NS * SH;
  static constexpr int X3 = X2 + NS * SH;
  static constexpr int X4 = X3 + NS * SG;
  static constexpr int X5 = X4 + NS * SH;
  static constexpr int OUT = X5 + NS * SH;
  static constexpr int DA = OUT + NS * 4;
  static constexpr int TOTAL = DA + NS * SH;  // floats
  // weight-gradient registers per thread
  static constexpr int NW1 = H * IN / NT;
  static constexpr int NW2 = H * H / NT;
  static constexpr int NW3 = (G * H + NT - 1) / NT;
  static constexpr int NV1 = COL ? (H * CIN + NT - 1) / NT : 1;
  static constexpr int NV2 = COL ? H * H / NT : 1;
  static constexpr int NV3 = COL ? (3 * H + NT - 1) / NT : 1;
};

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// out[s][o] = act(W[o] . in[s]) for o = hh, hh + 2, ... (W row-major [O][I] in global memory).
template <int I, int O, bool RELU>
__device__ __forceinline__ void layer_fwd(const float *__restrict__ W, const float *in_row, float *out_row, int hh) {
  float x[I];
#pragma unroll
  for (int i = 0; i < I; ++i) x[i] = in_row[i];
  for (int o = hh; o < O; o += 2) {
    const float4 *w4 = reinterpret_cast<const float4 *>(W + (size_t)o * I);
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < I / 4; ++i) {
      const float4 w = __ldg(w4 + i);
      acc = fmaf(w.x, x[4 * i + 0], acc);
      acc = fmaf(w.y, x[4 * i + 1], acc);
      acc = fmaf(w.z, x[4 * i + 2], acc);
      acc = fmaf(w.w, x[4 * i + 3], acc);
    }
    out_row[o] = RELU ? fmaxf(acc, 0.0f) : acc;
  }
}

// dx[s][i] = (mask ? act[s][i] > 0 : 1) * sum_o W[o][i] d[s][o] for i = hh, hh + 2, ... < I
// (W row-major with rows of LD >= I weights).
template <int I, int O, bool MASK, int LD = I>
__device__ __forceinline__ void layer_bwd(const float *__restrict__ W, const float *d_row, const float *act_row,
                                          float *dx_row, int hh) {
  float d[O];
#pragma unroll
  for (int o = 0; o < O; ++o) d[o] = d_row[o];
  for (int i = hh; i < I; i += 2) {
    float acc = 0.0f;
#pragma unroll
    for (int o = 0; o < O; ++o) acc = fmaf(__ldg(W + (size_t)o * LD + i), d[o], acc);
    if (MASK) acc = act_row[i] > 0.0f ? acc : 0.0f;
    dx_row[i] = acc;
  }
}

// acc[j] += sum_s D[s][o] A[s][i] for the weights w = tid + NT j (o = w / I, i = w % I) of an O x I layer.
template <int NJ, int O, int I>
__device__ __forceinline__ void accum_dw(float *acc, const float *D, int sd, const float *A, int sa, int tid) {
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int w = tid + NT * j;
    if (w < O * I) {
      const int o = w / I, i = w % I;
      float sum = 0.0f;
#pragma unroll 8
      for (int s = 0; s < NS; ++s) sum = fmaf(D[s * sd + o], A[s * sa + i], sum);
      acc[j] += sum;
    }
  }
}

template <int NJ, int NW>
__device__ __forceinline__ void flush_dw(float *acc, float *dst, int tid) {
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int w = tid + NT * j;
    if (w < NW && acc[j] != 0.0f) atomicAdd(dst + w, acc[j]);
    acc[j] = 0.0f;
  }
}

template <int IN, int G, bool COL, bool VD, int MODE>
__global__ void __launch_bounds__(NT, 2) k_field_fp32(const FieldArgs a) {
  using D = Dims<IN, G, COL, VD>;
  constexpr int CIN = D::CIN;
  constexpr int H = kHidden;
  extern __shared__ float sm[];
  float *X0 = sm + D::X0, *X1 = sm + D::X1, *X2 = sm + D::X2, *X3 = sm + D::X3, *X4 = sm + D::X4,
        *X5 = sm + D::X5, *OUT = sm + D::OUT, *DA = sm + D::DA;
  const int tid = threadIdx.x, s = tid & (NS - 1), hh = tid >> 6;
  const snk_state *st = a.state;
  const ModelDev &m = a.m;
  const GridParams &gp = m.grid;

  int64_t r0 = 0, r1 = st->slot_base[kMaxSlots];
  if (a.slot_only >= 0) {
    r0 = st->slot_base[a.slot_only];
    r1 = r0 + st->slot_count[a.slot_only];
  }
  if (r1 > a.S) r1 = a.S;
  const int64_t n_tiles = r1 > r0 ? (r1 - r0 + NS - 1) / NS : 0;

  float aW1[D::NW1], aW2[D::NW2], aW3[D::NW3], aV1[D::NV1], aV2[D::NV2], aV3[D::NV3];
  if (MODE == kBackward) {
#pragma unroll
    for (int j = 0; j < D::NW1; ++j) aW1[j] = 0.f;
#pragma unroll
    for (int j = 0; j < D::NW2; ++j) aW2[j] = 0.f;
#pragma unroll
    for (int j = 0; j < D::NW3; ++j) aW3[j] = 0.f;
#pragma unroll
    for (int j = 0; j < D::NV1; ++j) aV1[j] = 0.f;
#pragma unroll
    for (int j = 0; j < D::NV2; ++j) aV2[j] = 0.f;
#pragma unroll
    for (int j = 0; j < D::NV3; ++j) aV3[j] = 0.f;
  }
  int cur_slot = -1;

  auto flush = [&](int k) {
    float *g = a.grads + (int64_t)k * m.tile_params;
    flush_dw<D::NW1, H * IN>(aW1, g + m.w1, tid);
    flush_dw<D::NW2, H * H>(aW2, g + m.w2, tid);
    flush_dw<D::NW3, G * H>(aW3, g + m.w3, tid);
    if (COL) {
      float *c = a.grads + m.colour_base + (m.shared_colour ? 0 : (int64_t)k * m.colour_params);
      flush_dw<D::NV1, H * CIN>(aV1, c + m.v1, tid);
      flush_dw<D::NV2, H * H>(aV2, c + m.v2, tid);
      flush_dw<D::NV3, 3 * H>(aV3, c + m.v3, tid);
    }
  };

  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t ts = r0 + t * NS;
    const int slot = slot_of(st, ts);
    if (slot < 0) continue;  // padding tile (uniform across the block)
    if (MODE == kBackward && slot != cur_slot) {
      if (cur_slot >= 0) flush(cur_slot);
      cur_slot = slot;
    }
    const int64_t idx = ts + s;
    const bool valid = idx < (int64_t)st->slot_base[slot] + st->slot_count[slot] && idx < r1;
    const float *P = a.params + (int64_t)slot * m.tile_params;
    const float *Wg1 = P + m.w1, *Wg2 = P + m.w2, *Wg3 = P + m.w3;
    const float *C = a.params + m.colour_base + (m.shared_colour ? 0 : (int64_t)slot * m.colour_params);
    const float *V1 = C + m.v1, *V2 = C + m.v2, *V3 = C + m.v3;

    // ---- encode (or load features) ----
    float xyz[3] = {0.f, 0.f, 0.f};
    if (valid && a.feat_in == nullptr) {
#pragma unroll
      for (int q = 0; q < 3; ++q) xyz[q] = a.xyz[idx * 3 + q];
    }
    if (a.feat_in != nullptr) {
      for (int i = hh; i < IN; i += 2) X0[s * D::S0 + i] = valid ? a.feat_in[idx * IN + i] : 0.0f;
    } else {
      for (int l = hh; l < gp.L; l += 2) {
        const int N = gp.res[l];
        const bool dense = gp.dense[l] != 0;
        int ci[3];
        float fr[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) grid_cell(xyz[q], N, ci[q], fr[q]);
        const float2 *tab = reinterpret_cast<const float2 *>(P) + gp.offset[l];
        float f0 = 0.f, f1 = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
          const uint32_t e = grid_index(ci[0] + bx, ci[1] + by, ci[2] + bz, N, dense, (uint32_t)gp.T - 1u);
          const float w = (bx ? fr[0] : 1.0f - fr[0]) * (by ? fr[1] : 1.0f - fr[1]) * (bz ? fr[2] : 1.0f - fr[2]);
          if (valid) {
            const float2 v = __ldg(tab + e);
            f0 = fmaf(w, v.x, f0);
            f1 = fmaf(w, v.y, f1);
            if (a.idx_out) a.idx_out[(idx * gp.L + l) * 8 + c] = gp.offset[l] + e;
          }
        }
        X0[s * D::S0 + 2 * l] = f0;
        X0[s * D::S0 + 2 * l + 1] = f1;
        if (a.feat_out && valid) {
          a.feat_out[idx * IN + 2 * l] = f0;
          a.feat_out[idx * IN + 2 * l + 1] = f1;
        }
      }
    }
    if (VD && MODE != kEncodeOnly && hh == 0) {
      // colour input columns G .. G + 15: SH of the sample's ray direction
      float d[3] = {0.f, 0.f, 1.f}, v[16];
      if (valid) {
        const uint32_t r = a.smp_ray[idx];
#pragma unroll
        for (int q = 0; q < 3; ++q) d[q] = a.ray_od[(int64_t)(3 + q) * a.n_rays + r];
      }
      sh16(d[0], d[1], d[2], v);
#pragma unroll
      for (int j = 0; j < 16; ++j) X3[s * D::SG + G + j] = v[j];
    }
    __syncthreads();
    if (MODE == kEncodeOnly) continue;

    // ---- forward ----
    layer_fwd<IN, H, true>(Wg1, X0 + s * D::S0, X1 + s * D::SH, hh);
    __syncthreads();
    layer_fwd<H, H, true>(Wg2, X1 + s * D::SH, X2 + s * D::SH, hh);
    __syncthreads();
    layer_fwd<H, G, false>(Wg3, X2 + s * D::SH, X3 + s * D::SG, hh);
    __syncthreads();
    if (COL) {
      layer_fwd<CIN, H, true>(V1, X3 + s * D::SG, X4 + s * D::SH, hh);
      __syncthreads();
      layer_fwd<H, H, true>(V2, X4 + s * D::SH, X5 + s * D::SH, hh);
      __syncthreads();
      for (int o = hh; o < 3; o += 2) {
        const float4 *w4 = reinterpret_cast<const float4 *>(V3 + o * H);
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < H / 4; ++i) {
          const float4 w = __ldg(w4 + i);
          const float *x = X5 + s * D::SH + 4 * i;
          acc = fmaf(w.x, x[0], acc);
          acc = fmaf(w.y, x[1], acc);
          acc = fmaf(w.z, x[2], acc);
          acc = fmaf(w.w, x[3], acc);
        }
        OUT[s * 4 + 1 + o] = sigmoidf_(acc);
      }
    } else if (hh == 0) {
      for (int o = 0; o < 3; ++o) OUT[s * 4 + 1 + o] = sigmoidf_(X3[s * D::SG + 1 + o]);
    }
    if (hh == 0) OUT[s * 4 + 0] = expf(X3[s * D::SG + 0]);
    __syncthreads();

    if (MODE == kForward) {
      if (hh == 0 && valid)
        reinterpret_cast<float4 *>(a.sigma_rgb)[idx] =
            make_float4(OUT[s * 4 + 0], OUT[s * 4 + 1], OUT[s * 4 + 2], OUT[s * 4 + 3]);
      continue;
    }

    // ---- backward ----
    if (hh == 0) {
      float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) d = reinterpret_cast<const float4 *>(a.dsr)[idx];
      const float g0 = fminf(fmaxf(X3[s * D::SG + 0], -15.0f), 15.0f);
      const float r = OUT[s * 4 + 1], gg = OUT[s * 4 + 2], b = OUT[s * 4 + 3];
      OUT[s * 4 + 0] = d.x * expf(g0);
      OUT[s * 4 + 1] = d.y * r * (1.0f - r);
      OUT[s * 4 + 2] = d.z * gg * (1.0f - gg);
      OUT[s * 4 + 3] = d.w * b * (1.0f - b);
    }
    __syncthreads();
    if (COL) {
      // delta of c2 (into DA), then dV3 = delta3 (x) c2
      layer_bwd<H, 3, true>(V3, OUT + s * 4 + 1, X5 + s * D::SH, DA + s * D::SH, hh);
      accum_dw<D::NV3, 3, H>(aV3, OUT + 1, 4, X5, D::SH, tid);
      __syncthreads();
      // delta of c1 (into X5), dV2 = delta_c2 (x) c1
      layer_bwd<H, H, true>(V2, DA + s * D::SH, X4 + s * D::SH, X5 + s * D::SH, hh);
      accum_dw<D::NV2, H, H>(aV2, DA, D::SH, X4, D::SH, tid);
      __syncthreads();
      // delta of g (into DA) = V1^T delta_c1 + (dsigma term on g0), dV1 = delta_c1 (x) g
      layer_bwd<G, H, false, CIN>(V1, X5 + s * D::SH, nullptr, DA + s * D::SH, hh);
      accum_dw<D::NV1, H, CIN>(aV1, X5, D::SH, X3, D::SG, tid);
      __syncthreads();
      if (hh == 0) DA[s * D::SH + 0] += OUT[s * 4 + 0];
      __syncthreads();
    } else {
      if (hh == 0) {
        DA[s * D::SH + 0] = OUT[s * 4 + 0];
        for (int o = 1; o < G; ++o) DA[s * D::SH + o] = o < 4 ? OUT[s * 4 + o] : 0.0f;
      }
      __syncthreads();
    }
    // delta of h2 (into X4), dW3 = delta_g (x) h2
    layer_bwd<H, G, true>(Wg3, DA + s * D::SH, X2 + s * D::SH, X4 + s * D::SH, hh);
    accum_dw<D::NW3, G, H>(aW3, DA, D::SH, X2, D::SH, tid);
    __syncthreads();
    // delta of h1 (into X5), dW2 = delta_h2 (x) h1
    layer_bwd<H, H, true>(Wg2, X4 + s * D::SH, X1 + s * D::SH, X5 + s * D::SH, hh);
    accum_dw<D::NW2, H, H>(aW2, X4, D::SH, X1, D::SH, tid);
    __syncthreads();
    // dfeat (into DA), dW1 = delta_h1 (x) feat
    layer_bwd<IN, H, false>(Wg1, X5 + s * D::SH, nullptr, DA + s * D::SH, hh);
    accum_dw<D::NW1, H, IN>(aW1, X5, D::SH, X0, D::S0, tid);
    __syncthreads();

    // ---- hash-table scatter of dfeat (or write it out) ----
    if (!valid) continue;
    if (a.dfeat_out != nullptr) {
      for (int i = hh; i < IN; i += 2) a.dfeat_out[idx * IN + i] = DA[s * D::SH + i];
      continue;
    }
    float2 *gtab_base = reinterpret_cast<float2 *>(a.grads + (int64_t)slot * m.tile_params);
    for (int l = hh; l < gp.L; l += 2) {
      const int N = gp.res[l];
      const bool dense = gp.dense[l] != 0;
      int ci[3];
      float fr[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) grid_cell(xyz[q], N, ci[q], fr[q]);
      const float d0 = DA[s * D::SH + 2 * l], d1 = DA[s * D::SH + 2 * l + 1];
      float2 *gt = gtab_base + gp.offset[l];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
        const uint32_t e = grid_index(ci[0] + bx, ci[1] + by, ci[2] + bz, N, dense, (uint32_t)gp.T - 1u);
        const float w = (bx ? fr[0] : 1.0f - fr[0]) * (by ? fr[1] : 1.0f - fr[1]) * (bz ? fr[2] : 1.0f - fr[2]);
        atomicAdd(gt + e, make_float2(w * d0, w * d1));
      }
    }
  }
  if (MODE == kBackward && cur_slot >= 0) flush(cur_slot);
}

template <int IN, int G, bool COL, bool VD, int MODE>
cudaError_t launch_t(const FieldArgs &a, int sm_count, cudaStream_t st, int ctas_per_sm) {
  using D = Dims<IN, G, COL, VD>;
  const size_t smem = sizeof(float) * D::TOTAL;
  auto k = k_field_fp32<IN, G, COL, VD, MODE>;
  static std::atomic<uint32_t> attr_done{0};  // per instantiation: devices whose limit is set
  if (cudaError_t e = set_smem_limit(k, (int)smem, attr_done); e != cudaSuccess) return e;
  const int64_t max_tiles = (a.S + NS - 1) / NS;
  int64_t grid = (int64_t)sm_count * ctas_per_sm;
  if (grid > max_tiles) grid = max_tiles;
  if (grid <= 0) return cudaSuccess;
  k<<<(unsigned)grid, NT, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <int IN, int G, bool COL, bool VD>
cudaError_t launch_mode(const FieldArgs &a, int sm_count, cudaStream_t st, int c) {
  switch (a.mode) {
    case kEncodeOnly: return launch_t<IN, G, COL, VD, kEncodeOnly>(a, sm_count, st, c);
    case kForward: return launch_t<IN, G, COL, VD, kForward>(a, sm_count, st, c);
    default: return launch_t<IN, G, COL, VD, kBackward>(a, sm_count, st, c);
  }
}

template <int IN>
cudaError_t launch_in(const FieldArgs &a, int sm_count, cudaStream_t st, int c) {
  if (a.m.colour && a.m.view_dirs && a.mode != kEncodeOnly) {
    if (a.smp_ray == nullptr || a.ray_od == nullptr || a.n_rays < 1) return cudaErrorInvalidValue;
    return launch_mode<IN, 16, true, true>(a, sm_count, st, c);
  }
  if (a.m.colour) return launch_mode<IN, 16, true, false>(a, sm_count, st, c);
  return launch_mode<IN, 4, false, false>(a, sm_count, st, c);
}

// Thread per (sample, level): trilinear scatter-add of a feature gradient.
__global__ void k_encode_scatter(const FieldArgs a) {
  const GridParams &gp = a.m.grid;
  const int64_t n = a.S * gp.L;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = q / gp.L;
    const int l = (int)(q % gp.L);
    const int slot = slot_of(a.state, idx);
    if (slot < 0) continue;
    const int N = gp.res[l];
    const bool dense = gp.dense[l] != 0;
    int ci[3];
    float fr[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) grid_cell(a.xyz[idx * 3 + k], N, ci[k], fr[k]);
    const int in = a.m.in_dim;
    const float d0 = a.feat_in[idx * in + 2 * l], d1 = a.feat_in[idx * in + 2 * l + 1];
    float2 *gt = reinterpret_cast<float2 *>(a.grads + (int64_t)slot * a.m.tile_params) + gp.offset[l];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
      const uint32_t e = grid_index(ci[0] + bx, ci[1] + by, ci[2] + bz, N, dense, (uint32_t)gp.T - 1u);
      const float w = (bx ? fr[0] : 1.0f - fr[0]) * (by ? fr[1] : 1.0f - fr[1]) * (bz ? fr[2] : 1.0f - fr[2]);
      atomicAdd(gt + e, make_float2(w * d0, w * d1));
    }
  }
}

}  // namespace

cudaError_t launch_encode_scatter(const FieldArgs &a, cudaStream_t st) {
  const int64_t n = a.S * a.m.grid.L;
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_encode_scatter<<<(unsigned)blocks, 256, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_field_fp32(const FieldArgs &a, int sm_count, cudaStream_t st, const Tuning &tu) {
  const int c = tu.fp32_ctas;
  switch (a.m.in_dim) {
    case 8: return launch_in<8>(a, sm_count, st, c);
    case 16: return launch_in<16>(a, sm_count, st, c);
    case 32: return launch_in<32>(a, sm_count, st, c);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace snk
