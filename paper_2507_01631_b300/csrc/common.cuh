// Shared device-side definitions of libsnk (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "../../include/snk.h"

namespace snk {

constexpr int kHidden = 64;
constexpr int kMaxSlots = 4;
constexpr int kMaxViews = 256;
constexpr int kMaxLevels = 32;
constexpr int kSlotAlign = 128;   // slot-major sample ranges start on multiples of this
constexpr uint32_t kStatusOverflow = 1u;
constexpr uint32_t kStatusCheck = 2u;
constexpr uint32_t kStatusTimeout = 4u;

// Camera of one view as the kernels see it (binary64 coefficients).
struct DevView {
  int32_t kind, width, height, crop_r0, crop_c0, crop_h, crop_w, pad;
  double a[4], b[4];
  double off[5], scale[5];
  double coef[4][20];
  const float *crop;  // crop_h x crop_w x 3 binary32, or nullptr
};

// Window constants.  The binary32 values are the correctly rounded images of
// the binary64 descriptor (computed on the host), so that every discrete
// decision is a fixed IEEE binary32 sequence.
struct WinParams {
  double origin[3];
  double z_min, z_max;
  float win_hi[3];       // nx*Wt, ny*Ht, Z (window-local)
  float scene_lo[3], scene_hi[3];
  float split[2];        // interior planes x = Wt, y = Ht
  float inv_size[3];     // 1/Wt, 1/Ht, 1/Z
  int32_t nx, ny;
  int32_t slot[4];
  int32_t n_slots;
};

struct SamplerParams {
  int32_t K_ray, K_min, K_max, render;
  uint32_t seed, iteration;
  int32_t use_state_iteration;  // 1: the jitter key's second word is state->iteration
  int32_t occ_res;              // occupancy culling: cells per axis (0: none)
  const uint8_t *occ;           // [n_slots][occ_res^3] occupied flags, cell (x, y, z) at (z R + y) R + x
  int32_t mode;                 // kSampleSegments, kSampleUniform or kSamplePoints
};
// Sampler modes: the segmented sampler (Sec. 4.5; K bins per segment, delta = bin width); the
// NeRF-XL distribution the paper compares against (K_ray bins over the whole ray, each sample in
// the tile holding its point); point samples with both segment ends and delta_i = t_i - t_{i-1}.
constexpr int kSampleSegments = 0, kSampleUniform = 1, kSamplePoints = 2;


// Grid level table passed by value to kernels.
// Cell-major copies of the dense levels (mixed path): cell (x, y, z) of dense level l (x, y, z <
// N_l) is cell cell_off[l] + x + N_l (y + N_l z) of a slot's n_cells cells, and holds its 8 corners
// c = dx + 2 dy + 4 dz in order -- FP16 feature pairs (32 B a cell) for the forward's gather,
// binary32 gradient pairs (64 B a cell) for the backward's scatter.  dense_end: the first table
// entry after the last dense level (dense levels are the coarsest, a prefix of the levels).
struct GridParams {
  int32_t L, F, log2_T, T;
  int32_t res[kMaxLevels];
  int32_t dense[kMaxLevels];
  uint32_t offset[kMaxLevels];
  uint32_t cell_off[kMaxLevels];
  uint32_t n_cells;
  uint32_t dense_end;
};

// ---- exact binary32 / binary64 arithmetic (never contracted) --------------
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// ---- Philox-4x32-10 (Salmon et al. 2011) ---------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniform (x >> 8) * 2^-24, exact in binary32.
__device__ __forceinline__ float u32_to_unit(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }

// Stratified jitter of sample j of ray `ray`: counter (ray, j >> 2, 1, 0), lane j & 3.
__device__ __forceinline__ float jitter(uint32_t seed, uint32_t iteration, uint32_t ray, uint32_t j) {
  const uint4 r = philox4x32_10(make_uint4(ray, j >> 2, 1u, 0u), make_uint2(seed, iteration));
  const uint32_t lane = j & 3u;
  const uint32_t x = lane == 0 ? r.x : lane == 1 ? r.y : lane == 2 ? r.z : r.w;
  return u32_to_unit(x);
}

// Occupancy cell of a tile-local point l in [0, 1]^3 (binary32: c = min(floor(l R), R - 1)).
__device__ __forceinline__ uint32_t occ_cell(const float l[3], int R) {
  uint32_t c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int v = (int)floorf(fmul(l[a], (float)R));
    v = v < R - 1 ? v : R - 1;
    c[a] = (uint32_t)(v > 0 ? v : 0);
  }
  return (c[2] * (uint32_t)R + c[1]) * (uint32_t)R + c[0];
}

// ---- view-direction encoding -------------------------------------------------
// The 16 real spherical harmonics of degrees 0..3 of a unit direction (x, y, z), in the order
// (l, m) = (0, 0), (1, -1), (1, 0), (1, 1), (2, -2), ..., (3, 3), with the sign convention of the
// usual graphics tables (Instant-NGP's direction encoding); the constants are the normalisations
// sqrt((2l + 1) / 4 pi (l - |m|)! / (l + |m|)!) (times sqrt 2 for m != 0) folded with the
// polynomial coefficients.
__device__ __forceinline__ void sh16(float x, float y, float z, float (&v)[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  v[0] = 0.28209479177387814f;
  v[1] = -0.48860251190291987f * y;
  v[2] = 0.48860251190291987f * z;
  v[3] = -0.48860251190291987f * x;
  v[4] = 1.0925484305920792f * x * y;
  v[5] = -1.0925484305920792f * y * z;
  v[6] = 0.94617469575756008f * zz - 0.31539156525252005f;
  v[7] = -1.0925484305920792f * x * z;
  v[8] = 0.54627421529603959f * (xx - yy);
  v[9] = -0.59004358992664352f * y * (3.0f * xx - yy);
  v[10] = 2.8906114426405538f * x * y * z;
  v[11] = 0.45704579946446572f * y * (1.0f - 5.0f * zz);
  v[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);
  v[13] = 0.45704579946446572f * x * (1.0f - 5.0f * zz);
  v[14] = 1.4453057213202769f * z * (xx - yy);
  v[15] = 0.59004358992664352f * x * (3.0f * yy - xx);
}

// ---- NGP dense index / spatial hash ----------------------------------------
__device__ __forceinline__ uint32_t grid_index(uint32_t x, uint32_t y, uint32_t z, int N, bool dense, uint32_t Tmask) {
  if (dense) {
    const uint32_t n1 = (uint32_t)N + 1u;
    return x + y * n1 + z * n1 * n1;
  }
  return (x ^ (y * 2654435761u) ^ (z * 805459861u)) & Tmask;
}

// Cell of one axis at resolution N: g = x * N (binary32), i = min(floor(g), N - 1), frac = g - i.
__device__ __forceinline__ void grid_cell(float x, int N, int &i, float &frac) {
  const float g = fmul(x, (float)N);
  int c = (int)floorf(g);
  c = c < N - 1 ? c : N - 1;
  c = c > 0 ? c : 0;
  i = c;
  frac = fsub(g, (float)c);
}

// Slot of a slot-major sample index; -1 for padding.
__device__ __forceinline__ int slot_of(const snk_state *st, int64_t s) {
#pragma unroll
  for (int k = 0; k < kMaxSlots; ++k) {
    const int64_t b = st->slot_base[k];
    if (s >= b && s < b + (int64_t)st->slot_count[k]) return k;
  }
  return -1;
}

__device__ __forceinline__ void set_status(snk_state *st, uint32_t bit) { atomicOr(&st->status, bit); }

// ---- L2 residency of the tables and their gradients ---------------------------
// The FP16 tables the forward gathers from and the binary32 gradients the backward reduces into
// are re-used by every sample of their slot, while the sample streams (stored activations,
// features) pass through once: table and gradient accesses carry an evict-last L2 policy, the
// streams an evict-first one.
__device__ __forceinline__ uint64_t l2_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_keep_b32(const void *a, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ uint2 ld_keep_v2(const void *a, uint64_t pol) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void red_keep_v4(float *a, float x, float y, float z, float w, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(x), "f"(y), "f"(z),
               "f"(w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void red_keep_v2(float *a, float x, float y, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(x), "f"(y), "l"(pol) : "memory");
}

// ---- x-adjacent corner pairs -------------------------------------------------
// Corners (x, y, z) and (x + 1, y, z) of a cell have entries e0, e1.  When they
// form one aligned pair {2k, 2k + 1} -- the dense index with x + ... even, or the
// hash (whose x factor is 1) with x even -- one 8-byte load (FP16 features) or
// one 16-byte reduction (binary32 gradients) serves both; otherwise two accesses.
// The table and gradient blocks start on 16-byte boundaries (level sizes are
// multiples of 8 entries).

// v0 = table[e0], v1 = table[e1] (FP16 feature pairs), with L2 policy pol.
__device__ __forceinline__ void load_pair(const __half2 *tab, uint32_t e0, uint32_t e1, __half2 &v0, __half2 &v1,
                                          uint64_t pol) {
  uint32_t a, b;
  if ((e0 ^ e1) == 1u) {
    const uint2 u = ld_keep_v2(tab + (e0 & ~1u), pol);
    a = (e0 & 1u) ? u.y : u.x;
    b = (e0 & 1u) ? u.x : u.y;
  } else {
    a = ld_keep_b32(tab + e0, pol);
    b = ld_keep_b32(tab + e1, pol);
  }
  v0 = *reinterpret_cast<const __half2 *>(&a);
  v1 = *reinterpret_cast<const __half2 *>(&b);
}

// One level of the FP16 hash-grid gather (Sec. 4.1, NGP features): the cell of point x at
// resolution N (its fractions fr) and the feature pairs of its 8 corners, corner c at
// (x + (c & 1), y + ((c >> 1) & 1), z + ((c >> 2) & 1)); tab holds the level's entries.
__device__ __forceinline__ void gather_corners(const __half2 *tab, const float (&x)[3], int N, bool dense,
                                               uint32_t Tmask, __half2 (&hv)[8], float (&fr)[3], uint64_t pol) {
  int ci[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) grid_cell(x[q], N, ci[q], fr[q]);
#pragma unroll
  for (int c = 0; c < 8; c += 2)
    load_pair(tab, grid_index(ci[0], ci[1] + ((c >> 1) & 1), ci[2] + ((c >> 2) & 1), N, dense, Tmask),
              grid_index(ci[0] + 1, ci[1] + ((c >> 1) & 1), ci[2] + ((c >> 2) & 1), N, dense, Tmask), hv[c], hv[c + 1],
              pol);
}

// One dense level from its cell-major FP16 copy (GridParams): the cell of point x at resolution N
// (its fractions fr) and its 8 corner feature pairs, corner c = dx + 2 dy + 4 dz, in one 32-byte
// load.  level_cells: the level's first cell (32-byte aligned blocks).
__device__ __forceinline__ void gather_cell(const uint16_t *level_cells, const float (&x)[3], int N, __half2 (&hv)[8],
                                            float (&fr)[3], uint64_t pol) {
  int ci[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) grid_cell(x[q], N, ci[q], fr[q]);
  const uint32_t c = (uint32_t)ci[0] + (uint32_t)N * ((uint32_t)ci[1] + (uint32_t)N * (uint32_t)ci[2]);
  uint32_t r[8];
  asm volatile("ld.global.nc.L2::cache_hint.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "l"(level_cells + 16 * (size_t)c), "l"(pol));
#pragma unroll
  for (int q = 0; q < 8; ++q) hv[q] = *reinterpret_cast<const __half2 *>(&r[q]);
}

// Segmented sums over the lanes of a warp (all 32 lanes call it): the runs of consecutive lanes
// with equal `key` are the segments.  Afterwards the last lane of each run holds in v the sums of
// its run's values, and the function returns true there.  Steps stop once no lane's run reaches
// further back (a warp-uniform decision).
template <int NV>
__device__ __forceinline__ bool run_sums(float (&v)[NV], uint32_t key, int lane) {
  const uint32_t up = __shfl_up_sync(0xffffffffu, key, 1), dn = __shfl_down_sync(0xffffffffu, key, 1);
  const bool head = lane == 0 || up != key;
  const bool tail = lane == 31 || dn != key;
  const uint32_t heads = __ballot_sync(0xffffffffu, head);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of this lane's run
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const bool take = lane - off >= start;
    if (!__any_sync(0xffffffffu, take)) break;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float u = __shfl_up_sync(0xffffffffu, v[i], off);
      if (take) v[i] += u;
    }
  }
  return tail;
}

// Trilinear interpolation of the 8 corner feature pairs in binary32, corners summed in order.
__device__ __forceinline__ float2 interp_corners(const __half2 (&hv)[8], const float (&fr)[3]) {
  float f0 = 0.f, f1 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float w = ((c & 1) ? fr[0] : 1.0f - fr[0]) * ((c & 2) ? fr[1] : 1.0f - fr[1]) *
                    ((c & 4) ? fr[2] : 1.0f - fr[2]);
    const float2 v = __half22float2(hv[c]);
    f0 = fmaf(w, v.x, f0);
    f1 = fmaf(w, v.y, f1);
  }
  return make_float2(f0, f1);
}

// grad[e0] += w0 * d, grad[e1] += w1 * d (fire-and-forget reductions, L2 policy pol).
__device__ __forceinline__ void red_pair(float2 *grad, uint32_t e0, uint32_t e1, float w0, float w1, float2 d,
                                         uint64_t pol) {
  if ((e0 ^ e1) == 1u) {
    const bool odd = e0 & 1u;
    const float a = odd ? w1 : w0, b = odd ? w0 : w1;
    red_keep_v4(reinterpret_cast<float *>(grad + (e0 & ~1u)), a * d.x, a * d.y, b * d.x, b * d.y, pol);
  } else {
    red_keep_v2(reinterpret_cast<float *>(grad + e0), w0 * d.x, w0 * d.y, pol);
    red_keep_v2(reinterpret_cast<float *>(grad + e1), w1 * d.x, w1 * d.y, pol);
  }
}

// grad[e0] += a, grad[e1] += b (already weighted sums), merged when the two share an aligned pair.
__device__ __forceinline__ void red_pair_sums(float2 *grad, uint32_t e0, uint32_t e1, float2 a, float2 b,
                                              uint64_t pol) {
  if ((e0 ^ e1) == 1u) {
    float *q = reinterpret_cast<float *>(grad + (e0 & ~1u));
    if (e0 & 1u)
      red_keep_v4(q, b.x, b.y, a.x, a.y, pol);
    else
      red_keep_v4(q, a.x, a.y, b.x, b.y, pol);
  } else {
    red_keep_v2(reinterpret_cast<float *>(grad + e0), a.x, a.y, pol);
    red_keep_v2(reinterpret_cast<float *>(grad + e1), b.x, b.y, pol);
  }
}

// ---- E4M3 (OCP 8-bit float: sign, 4 exponent bits with bias 7, 3 mantissa bits,
// largest finite 448, no infinities) -----------------------------------------
// Two binary32 values to an E4M3 pair (lo in the low byte): round to nearest
// even, magnitudes beyond 448 saturate to 448.
__device__ __forceinline__ uint16_t e4m3x2_from_f32(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}
// An E4M3 pair as an FP16 pair (exact: every E4M3 value is an FP16 value).
__device__ __forceinline__ uint32_t f16x2_from_e4m3x2(uint16_t c) {
  uint32_t r;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(r) : "h"(c));
  return r;
}
// Per-slot scale of the E4M3 first-layer input: amax / 448 (1 for an all-zero slot).
__device__ __forceinline__ float e4m3_scale(uint32_t amax_bits) {
  const float amax = __uint_as_float(amax_bits);
  return amax > 0.f ? fdiv(amax, 448.0f) : 1.0f;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace snk
