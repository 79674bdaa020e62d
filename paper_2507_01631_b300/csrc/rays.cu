// S1 + S2: on-the-fly rays from satellite cameras, window acceptance, segment
// split, samples per segment, slot-major sample offsets and stratified sample
// placement.  Sec. 3 / 4.6 (rays are computed when needed, never stored for
// whole images), Sec. 4.4 (accept only rays
// whose tiles are all loaded), Sec. 4.5 (per-tile near/far pairs; each
// segment is sampled on its own so that its ends fall on tile faces).
//
// Every value that decides something discrete is a fixed sequence of IEEE
// operations written with explicit round-to-nearest intrinsics (no fused
// multiply-add): binary64 for the camera, binary32 for the box clipping,
// the segment bounds, the per-segment sample counts and the sample positions.
#include "camera.cuh"
#include "kernels.cuh"

namespace snk {

// NeRF-XL mode: sample j of the ray at t = t_in + (j + u) w (u = 0.5 when rendering).
__device__ __forceinline__ float uniform_t(float t_in, float w, const SamplerParams &smp, uint32_t iteration,
                                           uint32_t ray, uint32_t j) {
  const float u = smp.render ? 0.5f : jitter(smp.seed, iteration, ray, j);
  return fadd(t_in, fmul(fadd((float)j, u), w));
}

// Window tile (iy nx + ix) holding the point at t (a point on an interior plane goes to the lower tile).
__device__ __forceinline__ int point_tile(const float o[3], const float d[3], float t, const WinParams &win) {
  const int ix = (win.nx == 2 && fadd(o[0], fmul(t, d[0])) > win.split[0]) ? 1 : 0;
  const int iy = (win.ny == 2 && fadd(o[1], fmul(t, d[1])) > win.split[1]) ? 1 : 0;
  return iy * win.nx + ix;
}

// One thread per ray: camera -> (o, d) -> acceptance -> <= 3 segments -> K per segment.
__global__ void __launch_bounds__(512) k_rays(const DevView *__restrict__ views, int n_views, WinParams win, SamplerParams smp,
                       const uint32_t *__restrict__ pix, int B, int need_targets, float *__restrict__ ray_od,
                       uint8_t *__restrict__ ray_ok, uint8_t *__restrict__ seg_slot, float *__restrict__ seg_t,
                       uint32_t *__restrict__ seg_n, uint32_t *__restrict__ cnt, snk_state *state) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) {
    state->loss = 0.0f;
    state->nonfinite = 0u;  // non-finite-gradient flag of this step
  }
  if (r >= B) return;
  const uint32_t p = pix[r];
  const int v = (int)(p >> 24), row = (int)((p >> 12) & 0xFFFu), col = (int)(p & 0xFFFu);
  bool valid = v < n_views;
  if (valid && need_targets) {
    const DevView &cv = views[v];
    valid = cv.crop != nullptr && row >= cv.crop_r0 && row < cv.crop_r0 + cv.crop_h && col >= cv.crop_c0 &&
            col < cv.crop_c0 + cv.crop_w;
  }
  float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, -1.f};
  if (valid)
    pixel_ray(views[v], row, col, win, o, d);
  else
    set_status(state, kStatusCheck);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ray_od[(size_t)a * B + r] = o[a];
    ray_od[(size_t)(3 + a) * B + r] = d[a];
  }
  float inv[3];
  Slab sc;
  const bool ok = window_accepts(o, d, win, inv, sc) && valid;

  uint8_t s_slot[3] = {255, 255, 255};
  float s_t0[3] = {0.f, 0.f, 0.f}, s_t1[3] = {0.f, 0.f, 0.f};
  uint32_t s_n[3] = {0u, 0u, 0u};
  if (ok && smp.mode == kSampleUniform) {
    // K_ray bins over the whole scene interval; each sample belongs to the tile holding its point,
    // the samples of a tile are one run along the ray (x(t), y(t) are monotone) and one segment
    const float a = sc.t_in, b = sc.t_out;
    const uint32_t iteration = smp.use_state_iteration ? state->iteration : smp.iteration;
    const float w = fdiv(fsub(b, a), (float)smp.K_ray);
    int ns = -1, last = -1;
    for (int j = 0; j < smp.K_ray; ++j) {
      const float t = uniform_t(a, w, smp, iteration, (uint32_t)r, (uint32_t)j);
      const int tile = point_tile(o, d, t, win);
      if (tile != last) {
        if (++ns == 3) break;  // cannot happen: at most two interior planes are crossed
        last = tile;
        s_slot[ns] = (uint8_t)win.slot[tile];
        s_t0[ns] = a;
        s_t1[ns] = b;
      }
      s_n[ns] += 1u;
    }
  } else if (ok) {
    const float a = sc.t_in, b = sc.t_out;
    float cut[2] = {0.f, 0.f};
    int nc = 0;
    if (win.nx == 2 && d[0] != 0.0f) {
      const float tp = fmul(fsub(win.split[0], o[0]), inv[0]);
      if (a < tp && tp < b) cut[nc++] = tp;
    }
    if (win.ny == 2 && d[1] != 0.0f) {
      const float tp = fmul(fsub(win.split[1], o[1]), inv[1]);
      if (a < tp && tp < b) cut[nc++] = tp;
    }
    if (nc == 2 && cut[1] < cut[0]) {
      const float tmp = cut[0];
      cut[0] = cut[1];
      cut[1] = tmp;
    }
    float bnd[4] = {a, b, b, b};
    if (nc >= 1) bnd[1] = cut[0];
    if (nc == 2) bnd[2] = cut[1];
    bnd[1 + nc] = b;
    const float len_ray = fsub(b, a);
    int ns = 0;
    for (int j = 0; j < nc + 1; ++j) {
      const float lo_t = bnd[j], hi_t = bnd[j + 1];
      const float len = fsub(hi_t, lo_t);
      if (!(len > 0.0f)) continue;
      const float mid = fadd(lo_t, fmul(len, 0.5f));
      const int ix = (win.nx == 2 && fadd(o[0], fmul(mid, d[0])) > win.split[0]) ? 1 : 0;
      const int iy = (win.ny == 2 && fadd(o[1], fmul(mid, d[1])) > win.split[1]) ? 1 : 0;
      const float q = fdiv(len, len_ray);
      const float kf = fmul((float)smp.K_ray, q);
      int k = (int)rintf(kf);
      k = k < smp.K_min ? smp.K_min : k;
      k = k > smp.K_max ? smp.K_max : k;
      s_slot[ns] = (uint8_t)win.slot[iy * win.nx + ix];
      s_t0[ns] = lo_t;
      s_t1[ns] = hi_t;
      s_n[ns] = (uint32_t)k;
      ++ns;
    }
  }
  ray_ok[r] = ok ? 1 : 0;
  uint32_t c[kMaxSlots] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    seg_slot[(size_t)r * 3 + s] = s_slot[s];
    seg_t[((size_t)r * 3 + s) * 2 + 0] = s_t0[s];
    seg_t[((size_t)r * 3 + s) * 2 + 1] = s_t1[s];
    seg_n[(size_t)r * 3 + s] = s_n[s];
    if (s_slot[s] < kMaxSlots) c[s_slot[s]] += s_n[s];
  }
  for (int k = 0; k < win.n_slots; ++k) cnt[(size_t)k * B + r] = c[k];
  cnt[(size_t)kMaxSlots * B + r] = ok ? 1u : 0u;  // accepted-ray counter rides along as row 4
}

// ---- per-slot exclusive scan over rays ---------------------------------------
// Row k of cnt (k < n_slots) holds ray r's samples in slot k; row 4 the accepted flag.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanThreads * kScanPer;

__global__ void k_scan_local(const uint32_t *__restrict__ cnt, int B, int n_slots, uint32_t *__restrict__ excl,
                             uint32_t *__restrict__ block_tot) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const int row = (int)blockIdx.y < n_slots ? (int)blockIdx.y : kMaxSlots;  // rows 0..n_slots-1, then 4
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
  uint32_t v[kScanPer];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    v[i] = (base + i < B) ? cnt[(size_t)row * B + base + i] : 0u;
    sum += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = inc - sum + (warp > 0 ? warp_tot[warp - 1] : 0u);
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    if (base + i < B) excl[(size_t)row * B + base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == kScanThreads - 1) block_tot[(size_t)row * gridDim.x + blockIdx.x] = warp_tot[31];
}

// One block, one warp per row: scan the block totals of every row, place the
// slot ranges (each starting on a multiple of kSlotAlign), count accepted rays,
// check the sample capacity.
__global__ void k_scan_top(uint32_t *__restrict__ block_tot, int nb, int n_slots, int64_t cap, snk_state *state) {
  __shared__ uint32_t tot[kMaxSlots + 1];
  const int row = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (row < n_slots || row == kMaxSlots) {
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
      const int b = b0 + lane;
      const uint32_t v = b < nb ? block_tot[(size_t)row * nb + b] : 0u;
      uint32_t inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      if (b < nb) block_tot[(size_t)row * nb + b] = carry + inc - v;  // exclusive block base
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) tot[row] = carry;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t base = 0;
    uint32_t n = 0;
    for (int k = 0; k < kMaxSlots; ++k) {
      const uint32_t c = k < n_slots ? tot[k] : 0u;
      state->slot_base[k] = (uint32_t)base;
      state->slot_count[k] = c;
      n += c;
      base += c;
      base = (base + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
    }
    state->slot_base[kMaxSlots] = (uint32_t)base;
    state->n_accepted = tot[kMaxSlots];
    if ((int64_t)base > cap || base > 0xFFFFFFFFull) {
      set_status(state, kStatusCheck);
      for (int k = 0; k < kMaxSlots; ++k) state->slot_count[k] = 0u;
      state->slot_base[kMaxSlots] = 0u;
      state->n_samples = 0u;
    } else {
      state->n_samples = n;
    }
  }
}

// Warp per ray: segment offsets, then t, delta and tile-local xyz of every sample.
// Window-local lower corner of the tile of parameter slot k.
__device__ __forceinline__ void tile_lo(const WinParams &win, int k, float lo[3]) {
  int tile = 0;
  for (int q = 0; q < win.nx * win.ny; ++q)
    if (win.slot[q] == k) tile = q;
  const int ix = tile % win.nx, iy = tile / win.nx;
  lo[0] = ix ? win.split[0] : 0.0f;
  lo[1] = iy ? win.split[1] : 0.0f;
  lo[2] = 0.0f;
}

// Tile-local position in [0, 1]^3 of the point at t.
__device__ __forceinline__ void tile_local(const float o[3], const float d[3], float t, const float lo[3],
                                           const WinParams &win, float l[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p = fadd(o[a], fmul(t, d[a]));
    const float v = fmul(fsub(p, lo[a]), win.inv_size[a]);
    l[a] = fminf(fmaxf(v, 0.0f), 1.0f);
  }
}

// Candidate i of a segment (bin width w from t0; jitter index j0 + i along the ray):
// returns t and writes the tile-local position l in [0, 1]^3.
__device__ __forceinline__ float candidate(const float o[3], const float d[3], const float lo[3], const WinParams &win,
                                           const SamplerParams &smp, uint32_t iteration, uint32_t ray, uint32_t i,
                                           uint32_t j0, float w, float t0, float l[3]) {
  const float u = smp.render ? 0.5f : jitter(smp.seed, iteration, ray, j0 + i);
  const float t = fadd(t0, fmul(fadd((float)i, u), w));
  tile_local(o, d, t, lo, win, l);
  return t;
}

__device__ __forceinline__ bool occupied(const SamplerParams &smp, int slot, const float l[3]) {
  if (!smp.occ) return true;
  const size_t R3 = (size_t)smp.occ_res * smp.occ_res * smp.occ_res;
  return smp.occ[(size_t)slot * R3 + occ_cell(l, smp.occ_res)] != 0;
}

__global__ void __launch_bounds__(512) k_samples(const float *__restrict__ ray_od, const uint8_t *__restrict__ seg_slot,
                          const float *__restrict__ seg_t, const uint32_t *__restrict__ seg_n,
                          const uint32_t *__restrict__ excl, const uint32_t *__restrict__ block_tot, int nb, int B,
                          WinParams win, SamplerParams smp, const snk_state *__restrict__ state,
                          const uint32_t *__restrict__ seg_k, uint32_t *__restrict__ seg_off,
                          float *__restrict__ smp_t, float *__restrict__ smp_dt, float *__restrict__ smp_xyz,
                          uint32_t *__restrict__ smp_ray) {
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= B) return;
  const int r = warp;
  const uint32_t iteration = smp.use_state_iteration ? state->iteration : smp.iteration;
  float o[3], d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o[a] = ray_od[(size_t)a * B + r];
    d[a] = ray_od[(size_t)(3 + a) * B + r];
  }
  uint32_t j0 = 0;         // jitter index of the segment's first candidate along the ray
  float t_last = __int_as_float(0x7fffffff);  // points mode: t of the ray's previous sample (NaN: none)
  for (int s = 0; s < 3; ++s) {
    const int k = seg_slot[(size_t)r * 3 + s];
    const uint32_t n = seg_n[(size_t)r * 3 + s];                 // samples written
    const uint32_t nk = smp.occ ? seg_k[(size_t)r * 3 + s] : n;  // stratified candidates
    uint32_t off = 0;
    const bool live = k < kMaxSlots && n > 0 && state->slot_count[k] > 0;
    if (live) off = state->slot_base[k] + block_tot[(size_t)k * nb + r / kScanChunk] + excl[(size_t)k * B + r];
    if (lane == 0) seg_off[(size_t)r * 3 + s] = off;
    if (!live) {
      j0 += nk;
      continue;
    }
    const float t0 = seg_t[((size_t)r * 3 + s) * 2 + 0], t1 = seg_t[((size_t)r * 3 + s) * 2 + 1];
    // bin width: K bins per segment, K_ray bins over the ray (NeRF-XL), or K - 1 gaps (points)
    const float w = smp.mode == kSampleUniform ? fdiv(fsub(t1, t0), (float)smp.K_ray)
                    : smp.mode == kSamplePoints ? fdiv(fsub(t1, t0), (float)(nk - 1))
                                                : fdiv(fsub(t1, t0), (float)nk);
    float lo[3];
    tile_lo(win, k, lo);
    // the candidates in order; with culling only the occupied ones, compacted in order
    uint32_t written = 0;
    for (uint32_t i0 = 0; i0 < nk; i0 += 32) {
      const uint32_t i = i0 + lane;
      float t = 0.f, dt = w, l[3] = {0.f, 0.f, 0.f};
      bool keep = false;
      if (i < nk) {
        if (smp.mode == kSampleSegments) {
          t = candidate(o, d, lo, win, smp, iteration, (uint32_t)r, i, j0, w, t0, l);
        } else if (smp.mode == kSampleUniform) {
          t = uniform_t(t0, w, smp, iteration, (uint32_t)r, j0 + i);
          tile_local(o, d, t, lo, win, l);
        } else {
          t = i + 1 == nk ? t1 : fadd(t0, fmul((float)i, w));
          const float tp = i == 0 ? (t_last == t_last ? t_last : t) : fadd(t0, fmul((float)(i - 1), w));
          dt = fsub(t, tp);
          tile_local(o, d, t, lo, win, l);
        }
        keep = occupied(smp, k, l);
      }
      const uint32_t m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const size_t q = (size_t)off + written + __popc(m & ((1u << lane) - 1u));
        smp_t[q] = t;
        smp_dt[q] = dt;
#pragma unroll
        for (int a = 0; a < 3; ++a) smp_xyz[q * 3 + a] = l[a];
        if (smp_ray) smp_ray[q] = (uint32_t)r;
      }
      written += __popc(m);
    }
    if (smp.mode == kSamplePoints) t_last = t1;  // the segment's last point
    j0 += nk;
  }
}

// Occupancy culling, count pass (warp per ray; Sec. 4.1, the SAT-NGP coarse voxel grid): the
// stratified candidates of every segment are recomputed exactly as k_samples will place them and
// kept if their cell is occupied.  seg_k <- candidates, seg_n <- kept, cnt rows <- kept per slot.
__global__ void __launch_bounds__(512) k_cull_count(const float *__restrict__ ray_od, const uint8_t *__restrict__ seg_slot,
                                                    const float *__restrict__ seg_t, uint32_t *__restrict__ seg_n,
                                                    uint32_t *__restrict__ seg_k, uint32_t *__restrict__ cnt, int B,
                                                    WinParams win, SamplerParams smp,
                                                    const snk_state *__restrict__ state) {
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= B) return;
  const int r = warp;
  const uint32_t iteration = smp.use_state_iteration ? state->iteration : smp.iteration;
  float o[3], d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o[a] = ray_od[(size_t)a * B + r];
    d[a] = ray_od[(size_t)(3 + a) * B + r];
  }
  uint32_t j0 = 0;
  uint32_t c[kMaxSlots] = {0u, 0u, 0u, 0u};
  for (int s = 0; s < 3; ++s) {
    const int k = seg_slot[(size_t)r * 3 + s];
    const uint32_t nk = seg_n[(size_t)r * 3 + s];
    uint32_t kept = 0;
    if (k < kMaxSlots && nk > 0) {
      const float t0 = seg_t[((size_t)r * 3 + s) * 2 + 0], t1 = seg_t[((size_t)r * 3 + s) * 2 + 1];
      const float w = fdiv(fsub(t1, t0), (float)nk);
      float lo[3];
      tile_lo(win, k, lo);
      for (uint32_t i0 = 0; i0 < nk; i0 += 32) {
        const uint32_t i = i0 + lane;
        bool keep = false;
        if (i < nk) {
          float l[3];
          candidate(o, d, lo, win, smp, iteration, (uint32_t)r, i, j0, w, t0, l);
          keep = occupied(smp, k, l);
        }
        kept += __popc(__ballot_sync(0xffffffffu, keep));
      }
      c[k] += kept;
    }
    j0 += nk;
    if (lane == 0) {
      seg_k[(size_t)r * 3 + s] = nk;
      seg_n[(size_t)r * 3 + s] = kept;
    }
  }
  if (lane == 0)
    for (int k = 0; k < win.n_slots; ++k) cnt[(size_t)k * B + r] = c[k];
}

// ---- host launcher -------------------------------------------------------------
int scan_blocks(int B) { return (B + kScanChunk - 1) / kScanChunk; }

cudaError_t launch_sample_segments(const DevView *views, int n_views, const WinParams &win, const SamplerParams &smp,
                                   const uint32_t *pix, int B, int need_targets, const RayBuffers &rb, int64_t cap,
                                   snk_state *state, cudaStream_t st, const Tuning &tu) {
  if (B <= 0) return cudaSuccess;
  const int nt = tu.sampler_threads;
  k_rays<<<(B + nt - 1) / nt, nt, 0, st>>>(views, n_views, win, smp, pix, B, need_targets, rb.ray_od, rb.ray_ok,
                                          rb.seg_slot, rb.seg_t, rb.seg_n, rb.cnt, state);
  if (smp.occ) {
    if (!rb.seg_k) return cudaErrorInvalidValue;
    k_cull_count<<<(unsigned)(((int64_t)B * 32 + nt - 1) / nt), nt, 0, st>>>(rb.ray_od, rb.seg_slot, rb.seg_t, rb.seg_n,
                                                                           rb.seg_k, rb.cnt, B, win, smp, state);
    count_launches(1);
  }
  const int nb = scan_blocks(B);
  const dim3 g(nb, win.n_slots + 1);
  k_scan_local<<<g, kScanThreads, 0, st>>>(rb.cnt, B, win.n_slots, rb.excl, rb.block_tot);
  k_scan_top<<<1, 32 * (kMaxSlots + 1), 0, st>>>(rb.block_tot, nb, win.n_slots, cap, state);
  const int64_t threads = (int64_t)B * 32;
  k_samples<<<(unsigned)((threads + nt - 1) / nt), nt, 0, st>>>(rb.ray_od, rb.seg_slot, rb.seg_t, rb.seg_n, rb.excl,
                                                                rb.block_tot, nb, B, win, smp, state, rb.seg_k,
                                                                rb.seg_off, rb.smp_t, rb.smp_dt, rb.smp_xyz,
                                                                rb.smp_ray);
  count_launches(4);
  return cudaGetLastError();
}

}  // namespace snk
