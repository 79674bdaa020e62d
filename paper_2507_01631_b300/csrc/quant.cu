// E4M3 first-layer input of the mixed-precision path (the quantised variant of
// the density MLP's input; the encoding itself is Sec. 4.1, NGP).
//
// The per-tensor scale of a slot is amax / 448 over the slot's features of the
// current batch, so the features must all exist before the first layer can
// run: this pass gathers them (binary32, from the FP16 working copy of the
// tables, the same interpolation as the fused forward) into feat32 and reduces
// max |feature| per slot.  The tensor-core forward then reads feat32,
// quantises, and stores the codes for the backward.
#include "kernels.cuh"

namespace snk {
namespace {

// One thread per (sample, level): the level's two features, written as one
// float2 (a warp writes whole samples), and the warp's max |feature| folded
// into the slot's amax.  Slots start on multiples of 128 samples, so the
// samples of a warp (32 / L consecutive ones) share a slot or are padding.
__global__ void k_gather_amax(const FieldArgs a) {
  const GridParams &gp = a.m.grid;
  const int64_t n = a.S * gp.L;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the stride is a multiple of 32, so with n_round a multiple of 32 every lane of a warp
  // runs the same rounds (the warp-wide reductions below need all 32 lanes)
  const int64_t n_round = (n + 31) / 32 * 32;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_round; q += stride) {
    int slot = -1;
    float m = 0.f;
    if (q < n) {
      const int64_t idx = q / gp.L;
      const int l = (int)(q % gp.L);
      slot = slot_of(a.state, idx);
      if (slot >= 0) {
        const float x[3] = {a.xyz[idx * 3], a.xyz[idx * 3 + 1], a.xyz[idx * 3 + 2]};
        const __half2 *tab = reinterpret_cast<const __half2 *>(a.params_lp + (int64_t)slot * a.m.tile_params) +
                             gp.offset[l];
        __half2 hv[8];
        float fr[3];
        gather_corners(tab, x, gp.res[l], gp.dense[l] != 0, (uint32_t)gp.T - 1u, hv, fr, l2_keep());
        const float2 f = interp_corners(hv, fr);
        const float f0 = f.x, f1 = f.y;
        reinterpret_cast<float2 *>(a.feat32)[idx * gp.L + l] = make_float2(f0, f1);
        m = fmaxf(fabsf(f0), fabsf(f1));
      }
    }
    // non-negative binary32 values order like their bit patterns
    const uint32_t mb = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    const int lead = __ffs(__ballot_sync(0xffffffffu, slot >= 0)) - 1;
    const int sl = lead >= 0 ? __shfl_sync(0xffffffffu, slot, lead) : -1;
    if ((threadIdx.x & 31) == 0 && sl >= 0 && mb > 0u) atomicMax(a.amax + sl, mb);
  }
}

__global__ void k_quantize_e4m3(const float *x, int64_t n, float scale, uint8_t *codes) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 2 * i < n; i += stride) {
    const float lo = fdiv(x[2 * i], scale);
    const float hi = 2 * i + 1 < n ? fdiv(x[2 * i + 1], scale) : 0.f;
    const uint16_t c = e4m3x2_from_f32(lo, hi);
    codes[2 * i] = (uint8_t)(c & 0xffu);
    if (2 * i + 1 < n) codes[2 * i + 1] = (uint8_t)(c >> 8);
  }
}

}  // namespace

cudaError_t launch_gather_amax(const FieldArgs &a, int sm_count, cudaStream_t st) {
  const int64_t n = a.S * a.m.grid.L;
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)sm_count * 16) blocks = (int64_t)sm_count * 16;
  k_gather_amax<<<(unsigned)blocks, 256, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_quantize_e4m3(const float *x, int64_t n, float scale, uint8_t *codes, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = ((n + 1) / 2 + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_quantize_e4m3<<<(unsigned)blocks, 256, 0, st>>>(x, n, scale, codes);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace snk
