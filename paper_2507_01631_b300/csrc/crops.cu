// Image crops from ground tiles (Sec. 4.3) and the ray pool of a window,
// built on the device.
//
// Crops: every view projects the 8 corners of each tile of the window (the
// tile's box between z_min and z_max) to image coordinates with its camera
// model and takes the smallest pixel rectangle that contains them, widened by
// a margin and clipped to the image; a view's window crop is the union of its
// tiles' rectangles.  The synthetic cameras are localisation maps (pixel,
// height) -> ground, so a projection solves L(row, col, h) = (x, y) by Newton's
// method in binary64 with a forward-difference Jacobian (one-pixel steps),
// starting at the image centre, for a fixed number of iterations.
//
// Ray pool: the pixels of all window crops (view-major, then row-major inside
// the crop) whose rays the window accepts (Sec. 4.4), compacted in that order:
// flags per pixel and per-chunk counts, one scan over the chunk counts, then
// each chunk writes its accepted pixels at its offset in pixel order.  The
// acceptance is the sampler's own (camera.cuh), so a ray drawn from the pool
// is never rejected by the training step.
//
// Batches: B pixels drawn uniformly from the pool with Philox-4x32-10 (Salmon
// et al. 2011), counter (i / 4, 0, 0, 0) -- stream 0, the ray pick -- key
// (seed, iteration), word i % 4: index = (x >> 8) * n_pool >> 24.
#include "camera.cuh"
#include "kernels.cuh"

namespace snk {
namespace {

constexpr int kNewtonIters = 16;
constexpr int kChunkThreads = 256;
constexpr int kChunkPer = 16;
constexpr int kChunk = kChunkThreads * kChunkPer;  // pixels per chunk (one block)

// (row, col) with L(row, col, h) = (x, y); binary64, fixed op sequence.
__device__ void project(const DevView &v, double x, double y, double h, double &row, double &col) {
  row = dmul((double)v.height, 0.5);
  col = dmul((double)v.width, 0.5);
  for (int it = 0; it < kNewtonIters; ++it) {
    double x0, y0, xr, yr, xc, yc;
    localise(v, row, col, h, x0, y0);
    localise(v, dadd(row, 1.0), col, h, xr, yr);
    localise(v, row, dadd(col, 1.0), h, xc, yc);
    // J [dcol, drow]^T = [x - x0, y - y0]^T with J's columns (d/dcol, d/drow)
    const double j00 = dsub(xc, x0), j01 = dsub(xr, x0), j10 = dsub(yc, y0), j11 = dsub(yr, y0);
    const double det = dsub(dmul(j00, j11), dmul(j01, j10));
    if (!(det != 0.0)) break;
    const double ex = dsub(x, x0), ey = dsub(y, y0);
    const double dcol = ddiv(dsub(dmul(j11, ex), dmul(j01, ey)), det);
    const double drow = ddiv(dsub(dmul(j00, ey), dmul(j10, ex)), det);
    col = dadd(col, dcol);
    row = dadd(row, drow);
  }
}

// One block: thread 4 v + k handles tile k of the window in view v; then per-view unions.
__global__ void __launch_bounds__(256) k_crops(const DevView *__restrict__ views, int n_views, WinParams win, CropParams cp,
                        int32_t *__restrict__ tile_rects, int32_t *__restrict__ view_rects) {
  __shared__ int32_t rect[kMaxViews * 4][4];
  const int t = threadIdx.x;
  const int n_tiles = win.nx * win.ny;
  for (int u = t; u < n_views * 4; u += blockDim.x) {
    const int v = u >> 2, k = u & 3;
    int32_t r[4] = {0, 0, 0, 0};
    if (k < n_tiles) {
      const DevView &cv = views[v];
      const int ix = k % win.nx, iy = k / win.nx;
      double rmin = 1e300, rmax = -1e300, cmin = 1e300, cmax = -1e300;
      for (int c = 0; c < 8; ++c) {
        const double x = dadd(win.origin[0], dmul(cp.tile[0], (double)(ix + (c & 1))));
        const double y = dadd(win.origin[1], dmul(cp.tile[1], (double)(iy + ((c >> 1) & 1))));
        const double h = (c & 4) ? win.z_max : win.z_min;
        double row, col;
        project(cv, x, y, h, row, col);
        rmin = fmin(rmin, row);
        rmax = fmax(rmax, row);
        cmin = fmin(cmin, col);
        cmax = fmax(cmax, col);
      }
      // rows [floor(rmin) - margin, ceil(rmax) + margin) clipped to the image; empty if outside
      const double H = (double)cv.height, W = (double)cv.width;
      const double r0 = fmin(H, fmax(0.0, dsub(floor(rmin), (double)cp.margin)));
      const double c0 = fmin(W, fmax(0.0, dsub(floor(cmin), (double)cp.margin)));
      const double r1 = fmin(H, fmax(r0, dadd(ceil(rmax), (double)cp.margin)));
      const double c1 = fmin(W, fmax(c0, dadd(ceil(cmax), (double)cp.margin)));
      r[0] = (int32_t)r0;
      r[1] = (int32_t)c0;
      r[2] = (int32_t)(r1 - r0);
      r[3] = (int32_t)(c1 - c0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      rect[u][q] = r[q];
      tile_rects[u * 4 + q] = r[q];
    }
  }
  __syncthreads();
  for (int v = t; v < n_views; v += blockDim.x) {
    int32_t r0 = 1 << 30, c0 = 1 << 30, r1 = -1, c1 = -1;
    for (int k = 0; k < n_tiles; ++k) {
      const int32_t *q = rect[v * 4 + k];
      if (q[2] <= 0 || q[3] <= 0) continue;
      r0 = min(r0, q[0]);
      c0 = min(c0, q[1]);
      r1 = max(r1, q[0] + q[2]);
      c1 = max(c1, q[1] + q[3]);
    }
    const bool empty = r1 < 0;
    view_rects[v * 4 + 0] = empty ? 0 : r0;
    view_rects[v * 4 + 1] = empty ? 0 : c0;
    view_rects[v * 4 + 2] = empty ? 0 : r1 - r0;
    view_rects[v * 4 + 3] = empty ? 0 : c1 - c0;
  }
}

// base[v] = first pixel of view v in the pool enumeration (prefix of the crop areas).
__global__ void k_pool_base(const int32_t *__restrict__ vr, int n_views, int64_t *__restrict__ base) {
  if (threadIdx.x != 0) return;
  int64_t s = 0;
  for (int v = 0; v < n_views; ++v) {
    base[v] = s;
    const int32_t h = vr[v * 4 + 2], w = vr[v * 4 + 3];
    s += (h > 0 && w > 0) ? (int64_t)h * w : 0;
  }
  base[n_views] = s;
}

// Pixel g of the pool enumeration: its view (binary search over base) and packed id.
__device__ __forceinline__ uint32_t pixel_of(int64_t g, const int64_t *base, int n_views, const int32_t *vr, int &v,
                                             int &row, int &col) {
  int lo = 0, hi = n_views;  // base[lo] <= g < base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= g) lo = mid; else hi = mid;
  }
  v = lo;
  const int64_t q = g - base[v];
  const int w = vr[v * 4 + 3];
  row = vr[v * 4 + 0] + (int)(q / w);
  col = vr[v * 4 + 1] + (int)(q % w);
  return ((uint32_t)v << 24) | ((uint32_t)row << 12) | (uint32_t)col;
}

__global__ void __launch_bounds__(kChunkThreads) k_pool_flags(const DevView *__restrict__ views, int n_views, WinParams win,
                                                           const int32_t *__restrict__ vr, const int64_t *__restrict__ base,
                                                           uint8_t *__restrict__ flags, uint32_t *__restrict__ chunk_cnt) {
  const int64_t total = base[n_views];
  const int64_t g0 = (int64_t)blockIdx.x * kChunk;
  int cnt = 0;
  for (int j = 0; j < kChunkPer; ++j) {
    const int64_t g = g0 + j * kChunkThreads + threadIdx.x;
    bool ok = false;
    if (g < total) {
      int v, row, col;
      pixel_of(g, base, n_views, vr, v, row, col);
      float o[3], d[3], inv[3];
      Slab sc;
      pixel_ray(views[v], row, col, win, o, d);
      ok = window_accepts(o, d, win, inv, sc);
      flags[g] = ok ? 1 : 0;
    }
    cnt += __syncthreads_count(ok);
  }
  if (threadIdx.x == 0) chunk_cnt[blockIdx.x] = (uint32_t)cnt;
}

// One block: exclusive scan of the chunk counts.
// n_pool = min(total, cap); total = all accepted pixels (the caller compares the two).
__global__ void k_pool_scan(uint32_t *__restrict__ chunk_cnt, int n_chunks, int64_t cap, uint32_t *__restrict__ n_pool,
                            uint32_t *__restrict__ total) {
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < n_chunks; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    const uint32_t x = b < n_chunks ? chunk_cnt[b] : 0u;
    uint32_t incl = x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    if (w == 0) {
      const int nw = blockDim.x >> 5;
      uint32_t s = lane < nw ? warp_sum[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      if (lane < nw) warp_sum[lane] = s;
    }
    __syncthreads();
    const uint32_t before = carry + (w > 0 ? warp_sum[w - 1] : 0u) + incl - x;
    if (b < n_chunks) chunk_cnt[b] = before;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *n_pool = (int64_t)carry > cap ? (uint32_t)cap : carry;
    *total = carry;
  }
}

__global__ void __launch_bounds__(kChunkThreads) k_pool_write(int n_views, const int32_t *__restrict__ vr,
                                                           const int64_t *__restrict__ base,
                                                           const uint8_t *__restrict__ flags,
                                                           const uint32_t *__restrict__ chunk_off, int64_t cap,
                                                           uint32_t *__restrict__ pool) {
  __shared__ uint32_t warp_cnt[kChunkThreads / 32];
  const int64_t total = base[n_views];
  const int64_t g0 = (int64_t)blockIdx.x * kChunk;
  if (g0 >= total) return;
  uint32_t off = chunk_off[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = 0; j < kChunkPer; ++j) {
    const int64_t g = g0 + j * kChunkThreads + threadIdx.x;
    const bool ok = g < total && flags[g] != 0;
    const uint32_t m = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) warp_cnt[w] = __popc(m);
    __syncthreads();
    uint32_t before = off;
    for (int k = 0; k < w; ++k) before += warp_cnt[k];
    before += __popc(m & ((1u << lane) - 1u));
    if (ok && (int64_t)before < cap) {
      int v, row, col;
      pool[before] = pixel_of(g, base, n_views, vr, v, row, col);
    }
    uint32_t add = 0;
    for (int k = 0; k < kChunkThreads / 32; ++k) add += warp_cnt[k];
    off += add;
    __syncthreads();
  }
}

__global__ void k_draw(const uint32_t *__restrict__ pool, const uint32_t *__restrict__ n_pool, int B, uint32_t seed,
                       uint32_t iteration, uint32_t *__restrict__ pix) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const uint64_t n = *n_pool;
  if (n == 0) {
    pix[i] = 0xFFFFFFFFu;  // no view: the step rejects the ray and reports it
    return;
  }
  const uint4 r = philox4x32_10(make_uint4((uint32_t)(i >> 2), 0u, 0u, 0u), make_uint2(seed, iteration));
  const int lane = i & 3;
  const uint32_t x = lane == 0 ? r.x : lane == 1 ? r.y : lane == 2 ? r.z : r.w;
  pix[i] = pool[(((uint64_t)(x >> 8)) * n) >> 24];
}

}  // namespace

cudaError_t launch_crops(const DevView *views, int n_views, const WinParams &win, const CropParams &cp,
                         int32_t *tile_rects, int32_t *view_rects, cudaStream_t st) {
  k_crops<<<1, 256, 0, st>>>(views, n_views, win, cp, tile_rects, view_rects);
  count_launches(1);
  return cudaGetLastError();
}

int64_t pool_chunks(int64_t max_pixels) { return (max_pixels + kChunk - 1) / kChunk; }

cudaError_t launch_ray_pool(const DevView *views, int n_views, const WinParams &win, const int32_t *view_rects,
                            int64_t *base, int64_t max_pixels, uint8_t *flags, uint32_t *chunk_cnt, uint32_t *pool,
                            int64_t cap, uint32_t *n_pool, cudaStream_t st) {
  const int64_t nc = pool_chunks(max_pixels);
  if (nc <= 0 || nc > (1 << 30)) return cudaErrorInvalidValue;
  k_pool_base<<<1, 32, 0, st>>>(view_rects, n_views, base);
  k_pool_flags<<<(unsigned)nc, kChunkThreads, 0, st>>>(views, n_views, win, view_rects, base, flags, chunk_cnt);
  k_pool_scan<<<1, 1024, 0, st>>>(chunk_cnt, (int)nc, cap, n_pool, n_pool + 1);
  k_pool_write<<<(unsigned)nc, kChunkThreads, 0, st>>>(n_views, view_rects, base, flags, chunk_cnt, cap, pool);
  count_launches(4);
  return cudaGetLastError();
}

cudaError_t launch_draw(const uint32_t *pool, const uint32_t *n_pool, int B, uint32_t seed, uint32_t iteration,
                        uint32_t *pix, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_draw<<<(B + 255) / 256, 256, 0, st>>>(pool, n_pool, B, seed, iteration, pix);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace snk
