// Diagnostic: the rate at which this GPU retires fire-and-forget float reductions to random
// addresses of an L2-resident table -- the peak against which the training step's hash-table
// gradient scatter (S7c: 8 corner updates per sample and level) is reported.  Nothing else
// runs in the kernel: one reduction per iteration, a full-occupancy grid of grid-stride
// threads, addresses from a multiplicative integer hash of the operation index spread
// uniformly over the table's 16-byte slots.
#include "kernels.cuh"

namespace snk {
namespace {

// Slot of operation i: Knuth's multiplicative hash of (i + seed) (the 64-bit golden-ratio
// multiplier, high bits folded down), scaled onto [0, n16).
__device__ __forceinline__ uint32_t probe_slot(uint64_t i, uint32_t seed, uint32_t n16) {
  uint64_t x = (i + seed) * 0x9E3779B97F4A7C15ull;
  x ^= x >> 29;
  return (uint32_t)(((x >> 32) * (uint64_t)n16) >> 32);
}

// WIDTH = 16: one red.global.add.v4.f32 (a whole 16-byte slot); WIDTH = 8: one
// red.global.add.v2.f32 on the slot's first or second half (the parity of i).
template <int WIDTH>
__global__ void __launch_bounds__(256) k_red_probe(float *table, uint32_t n16, int64_t n_ops, uint32_t seed) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_ops; i += stride) {
    const uint32_t s = probe_slot((uint64_t)i, seed, n16);
    float *q = table + (size_t)s * 4;
    if (WIDTH == 16) {
      asm volatile("red.global.add.v4.f32 [%0], {%1, %1, %1, %1};" ::"l"(q), "f"(1.0f) : "memory");
    } else {
      q += 2 * (i & 1);
      asm volatile("red.global.add.v2.f32 [%0], {%1, %1};" ::"l"(q), "f"(1.0f) : "memory");
    }
  }
}

}  // namespace

cudaError_t launch_red_probe(float *table, int64_t n16, int64_t n_ops, int width, uint32_t seed, int sm_count,
                             cudaStream_t st) {
  if (n16 < 1 || n16 > 0xFFFFFFFFll || n_ops < 0 || (width != 8 && width != 16)) return cudaErrorInvalidValue;
  if (n_ops == 0) return cudaSuccess;
  const int blocks = sm_count * 8;  // 2048 threads a SM: full occupancy at 256 threads a block
  if (width == 16)
    k_red_probe<16><<<blocks, 256, 0, st>>>(table, (uint32_t)n16, n_ops, seed);
  else
    k_red_probe<8><<<blocks, 256, 0, st>>>(table, (uint32_t)n16, n_ops, seed);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace snk
