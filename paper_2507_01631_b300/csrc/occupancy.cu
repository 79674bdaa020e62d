// Occupancy grid of each tile (Sec. 4.1: SAT-NGP culls the samples that fall
// in empty space using a coarse voxel grid).  The update follows the usual
// rule of such grids: every cell of a slot's R^3 grid gets one density
// sample at a random point inside it, evaluated with the slot's own field
// (the same field kernels as a training step), the cell's density becomes
// max(decay x density, sigma), and a cell is occupied when its density
// exceeds min(threshold, mean density of the slot's grid).
//
// Points: cell (x, y, z) of slot k at index (z R + y) R + x; u = three words
// of Philox-4x32-10 with counter (cell, k, 3, 0) -- stream 3 -- and key (seed,
// step), each (w >> 8) 2^-24; the point is (cell + u) x (1 / R) per axis in
// binary32.  The mean is a fixed-order sum (per-block partial sums, then the
// blocks in order), so a threshold decision does not depend on timing.
#include "kernels.cuh"

namespace snk {
namespace {

constexpr int kOccThreads = 256;

__global__ void k_occ_points(int n_slots, int R, uint32_t seed, uint32_t step, float *__restrict__ xyz,
                             uint32_t *__restrict__ ray, snk_state *__restrict__ state) {
  const int64_t R3 = (int64_t)R * R * R;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    for (int k = 0; k <= kMaxSlots; ++k) state->slot_base[k] = (uint32_t)((k < n_slots ? k : n_slots) * R3);
    for (int k = 0; k < kMaxSlots; ++k) state->slot_count[k] = k < n_slots ? (uint32_t)R3 : 0u;
  }
  if (i >= n_slots * R3) return;
  const int k = (int)(i / R3);
  const uint32_t cell = (uint32_t)(i % R3);
  const uint4 w = philox4x32_10(make_uint4(cell, (uint32_t)k, 3u, 0u), make_uint2(seed, step));
  const uint32_t c[3] = {cell % (uint32_t)R, (cell / (uint32_t)R) % (uint32_t)R, cell / ((uint32_t)R * R)};
  const uint32_t u[3] = {w.x, w.y, w.z};
  const float inv = fdiv(1.0f, (float)R);
#pragma unroll
  for (int a = 0; a < 3; ++a) xyz[i * 3 + a] = fmul(fadd((float)c[a], u32_to_unit(u[a])), inv);
  ray[i] = 0u;
}

// density <- max(decay density, sigma); per-block partial sums of the new densities
__global__ void __launch_bounds__(kOccThreads) k_occ_ema(int64_t n, const float *__restrict__ sigma_rgb, float decay,
                                                         float *__restrict__ density, float *__restrict__ partial) {
  __shared__ float ws[kOccThreads / 32];
  const int64_t i = (int64_t)blockIdx.x * kOccThreads + threadIdx.x;
  float d = 0.f;
  if (i < n) {
    d = fmaxf(fmul(decay, density[i]), sigma_rgb[i * 4]);
    density[i] = d;
  }
  float s = d;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int q = 0; q < kOccThreads / 32; ++q) t += ws[q];
    partial[blockIdx.x] = t;
  }
}

// one thread per slot: thr[k] = min(threshold, mean of slot k) from the partial sums in order
__global__ void k_occ_mean(const float *__restrict__ partial, int blocks_per_slot, int n_slots, int64_t R3,
                           float threshold, float *__restrict__ thr) {
  const int k = threadIdx.x;
  if (k >= n_slots) return;
  double s = 0.0;
  for (int b = 0; b < blocks_per_slot; ++b) s += (double)partial[(int64_t)k * blocks_per_slot + b];
  const float mean = (float)(s / (double)R3);
  thr[k] = fminf(threshold, mean);
}

__global__ void k_occ_binarize(int64_t n, int64_t R3, const float *__restrict__ density, const float *__restrict__ thr,
                               uint8_t *__restrict__ occ) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  occ[i] = density[i] > thr[i / R3] ? 1 : 0;
}

}  // namespace

cudaError_t launch_occ_points(int n_slots, int R, uint32_t seed, uint32_t step, float *xyz, uint32_t *ray,
                              snk_state *state, cudaStream_t st) {
  const int64_t n = (int64_t)n_slots * R * R * R;
  k_occ_points<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_slots, R, seed, step, xyz, ray, state);
  count_launches(1);
  return cudaGetLastError();
}

int64_t occ_partials(int n_slots, int R) {
  const int64_t R3 = (int64_t)R * R * R;
  return (int64_t)n_slots * ((R3 + kOccThreads - 1) / kOccThreads);
}

cudaError_t launch_occ_update(int n_slots, int R, const float *sigma_rgb, float decay, float threshold,
                              float *density, uint8_t *occ, float *partial, float *thr, cudaStream_t st) {
  const int64_t R3 = (int64_t)R * R * R;
  const int64_t n = (int64_t)n_slots * R3;
  const int bps = (int)(R3 / kOccThreads);  // R a multiple of 8: R^3 a multiple of 512
  k_occ_ema<<<(unsigned)(n / kOccThreads), kOccThreads, 0, st>>>(n, sigma_rgb, decay, density, partial);
  k_occ_mean<<<1, 32, 0, st>>>(partial, bps, n_slots, R3, threshold, thr);
  k_occ_binarize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, R3, density, thr, occ);
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace snk
