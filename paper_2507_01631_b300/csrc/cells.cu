// Cell-major copies of the dense hash-grid levels (Sec. 4.1, NGP's dense levels: index x + y (N+1)
// + z (N+1)^2) for the mixed-precision field kernels.
//
// The forward gathers, for each sample and level, the 8 corners of its cell.  At a dense level
// those are 8 table entries in 4 x-adjacent pairs, half of them straddling an aligned pair: ~6
// scattered loads.  The cell-major copy stores each cell's 8 FP16 corner pairs in one 32-byte
// block, so the gather is one 32-byte load.  k_cells_copy writes it from the FP16 working copy
// before a forward.
//
// The backward adds w_c x dfeat into the 8 corners of each sample's cell.  At a dense level it
// adds into a cell-major binary32 accumulator (a cell's 8 corner pairs in one 64-byte block: four
// 16-byte reductions, after the scatter warps have summed the samples of a warp that share the
// cell); k_cells_fold then adds every corner of every cell into its vertex's table gradient and
// clears the accumulator (zero between steps).  The values and the sum they form are the same;
// only the order of the float additions differs.
#include "kernels.cuh"

namespace snk {
namespace {

// The dense level holding cell c of a slot's cell block (dense levels are a prefix of the levels).
__device__ __forceinline__ int cell_level(const GridParams &gp, uint32_t c) {
  int l = 0;
  for (int k = 1; k < gp.L; ++k)
    if (gp.dense[k] && gp.cell_off[k] <= c) l = k;
  return l;
}

__global__ void k_cells_copy(const uint16_t *__restrict__ params_lp, int64_t tile_params, GridParams gp,
                             int n_slots, uint16_t *__restrict__ cells) {
  const int64_t total = (int64_t)n_slots * gp.n_cells;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(j / gp.n_cells);
    const uint32_t c = (uint32_t)(j - (int64_t)slot * gp.n_cells);
    const int l = cell_level(gp, c);
    const uint32_t N = (uint32_t)gp.res[l], n1 = N + 1u, k = c - gp.cell_off[l];
    const uint32_t x = k % N, y = (k / N) % N, z = k / (N * N);
    const uint32_t *tab = reinterpret_cast<const uint32_t *>(params_lp + (int64_t)slot * tile_params) + gp.offset[l];
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      w[q] = __ldg(tab + (x + (q & 1)) + (y + ((q >> 1) & 1)) * n1 + (z + ((q >> 2) & 1)) * n1 * n1);
    uint4 *dst = reinterpret_cast<uint4 *>(cells) + 2 * j;
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

__global__ void k_cells_fold(float *__restrict__ cell_grad, float *__restrict__ grads, int64_t tile_params,
                             GridParams gp, int n_slots) {
  const int64_t total = (int64_t)n_slots * gp.dense_end;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(j / gp.dense_end);
    const uint32_t e = (uint32_t)(j - (int64_t)slot * gp.dense_end);
    int l = 0;
    for (int k = 1; k < gp.L; ++k)
      if (gp.dense[k] && gp.offset[k] <= e) l = k;
    const uint32_t N = (uint32_t)gp.res[l], n1 = N + 1u, k = e - gp.offset[l];
    if (k >= n1 * n1 * n1) continue;  // padding entries of the level
    const int x = (int)(k % n1), y = (int)((k / n1) % n1), z = (int)(k / (n1 * n1));
    float2 sum = make_float2(0.f, 0.f);
    float *cg = cell_grad + ((int64_t)slot * gp.n_cells + gp.cell_off[l]) * 16;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      // the vertex is corner q of the cell whose lower corner is (x, y, z) - offset(q)
      const int cx = x - (q & 1), cy = y - ((q >> 1) & 1), cz = z - ((q >> 2) & 1);
      if (cx < 0 || cy < 0 || cz < 0 || cx >= (int)N || cy >= (int)N || cz >= (int)N) continue;
      float2 *p = reinterpret_cast<float2 *>(cg + ((int64_t)cx + (int64_t)N * (cy + (int64_t)N * cz)) * 16) + q;
      const float2 v = *p;
      sum.x += v.x;
      sum.y += v.y;
      *p = make_float2(0.f, 0.f);
    }
    if (sum.x != 0.f || sum.y != 0.f) {
      float2 *g = reinterpret_cast<float2 *>(grads + (int64_t)slot * tile_params) + e;
      const float2 o = *g;
      *g = make_float2(o.x + sum.x, o.y + sum.y);
    }
  }
}

}  // namespace

cudaError_t launch_cells_copy(const uint16_t *params_lp, int64_t tile_params, const GridParams &gp, int n_slots,
                              uint16_t *cells, int sm_count, cudaStream_t st) {
  if (gp.n_cells == 0) return cudaSuccess;
  const int64_t total = (int64_t)n_slots * gp.n_cells;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)sm_count * 8) blocks = (int64_t)sm_count * 8;
  k_cells_copy<<<(unsigned)blocks, 256, 0, st>>>(params_lp, tile_params, gp, n_slots, cells);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_cells_fold(float *cell_grad, float *grads, int64_t tile_params, const GridParams &gp, int n_slots,
                              int sm_count, cudaStream_t st) {
  if (gp.n_cells == 0) return cudaSuccess;
  const int64_t total = (int64_t)n_slots * gp.dense_end;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)sm_count * 8) blocks = (int64_t)sm_count * 8;
  k_cells_fold<<<(unsigned)blocks, 256, 0, st>>>(cell_grad, grads, tile_params, gp, n_slots);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace snk
