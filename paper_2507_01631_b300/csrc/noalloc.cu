// snk_sample_segments_static: the ray / segment / sample stage for callers that
// cannot allocate device memory.  Some hosts own every byte of device memory
// themselves (a framework's caching allocator, a real-time renderer with a
// fixed budget, an embedding where the CUDA context is shared and cudaMalloc
// would synchronise or is forbidden).  They can pass their own input and
// output buffers but cannot let the library call cudaMalloc for its
// workspace, and cannot create an snk_ctx (which allocates).
//
// This entry point keeps its scratch -- the per-slot sample counts, their scans,
// the scan-block totals and the device copy of the cameras -- in one
// file-scope __device__ array of fixed size, present on every GPU that loads
// the library until the process exits.  It calls no cudaMalloc, cudaFree or
// other allocating routine.  It runs the same kernels as snk_sample_segments.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "kernels.cuh"

namespace snk {
namespace {

constexpr int kStaticMaxRays = 65536;                        // largest batch this entry point accepts
constexpr int kStaticMaxScanBlocks = kStaticMaxRays / 1024;  // >= scan blocks of any accepted batch
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kViewsBytes = align_up(sizeof(DevView) * kMaxViews);
constexpr size_t kRowsBytes = align_up(sizeof(uint32_t) * 5 * (size_t)kStaticMaxRays);
constexpr size_t kTotBytes = align_up(sizeof(uint32_t) * 5 * (size_t)kStaticMaxScanBlocks);
constexpr size_t kScratchBytes = kViewsBytes + 2 * kRowsBytes + kTotBytes;  // about 2.8 MB

// The scratch.  Host code must not pass g_scratch itself to a kernel: in host
// code the name stands for a host-side shadow, not a device address.  The
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_scratch_dev[kMaxDevices] = {nullptr};
DevView g_views_host[kMaxViews];  // host staging, guarded by g_mutex

int fail(char *err, int err_len, int code, const char *msg) {
  if (err && err_len > 0) snprintf(err, (size_t)err_len, "%s", msg);
  return code;
}

}  // namespace
}  // namespace snk

extern "C" int snk_sample_segments_static(const snk_window *win, const snk_camera *cams, int n_views,
                                          const uint32_t *pix, int B, const snk_sampler *sampler, float *ray_od,
                                          uint8_t *ray_ok, uint8_t *seg_slot, float *seg_t, uint32_t *seg_n,
                                          uint32_t *seg_off, float *smp_t, float *smp_dt, float *smp_xyz,
                                          int64_t cap, snk_state *state, snk_stream_t stream, char *err,
                                          int err_len) {
  using namespace snk;
  if (err && err_len > 0) err[0] = '\0';
  if (B < 0 || B > kStaticMaxRays)
    return fail(err, err_len, SNK_ERR_INVALID_ARG,
                "snk_sample_segments_static: B must be in 0..65536 (the fixed scratch holds 65536 rays)");
  if (!win || !sampler || !cams || n_views < 1 || n_views > kMaxViews)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: NULL descriptor or 1..256 views");
  if (B > 0 && (!pix || !ray_od || !ray_ok || !seg_slot || !seg_t || !seg_n || !seg_off || !smp_t || !smp_dt ||
                !smp_xyz || !state))
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: NULL buffer");
  if ((win->nx != 1 && win->nx != 2) || (win->ny != 1 && win->ny != 2))
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: window nx, ny must be 1 or 2");
  const int n_slots = win->nx * win->ny;
  int seen = 0;
  for (int q = 0; q < n_slots; ++q) {
    if (win->slot[q] < 0 || win->slot[q] >= n_slots || ((seen >> win->slot[q]) & 1))
      return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: slot[] is not a permutation");
    seen |= 1 << win->slot[q];
  }
  for (int a = 0; a < 3; ++a)
    if (!(win->tile_size[a] > 0.0) || !(win->scene_hi[a] > win->scene_lo[a]))
      return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: empty tile or scene box");
  if (sampler->K_min < 1 || sampler->K_max < sampler->K_min || sampler->K_max > 4096 || sampler->K_ray < 1 ||
      sampler->K_ray > 4096)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: bad K_ray / K_min / K_max");
  if (sampler->occ_res != 0 || sampler->occupancy != nullptr)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: no occupancy culling (no scratch for it)");
  for (int v = 0; v < n_views; ++v)
    if (cams[v].kind != SNK_CAM_AFFINE && cams[v].kind != SNK_CAM_RPC3)
      return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: unknown camera kind");

  // binary32 window constants: correctly rounded from the binary64 descriptor
  WinParams wp;
  memset(&wp, 0, sizeof(wp));
  for (int a = 0; a < 3; ++a) wp.origin[a] = win->origin[a];
  wp.z_min = win->origin[2];
  wp.z_max = win->origin[2] + win->tile_size[2];
  wp.win_hi[0] = (float)(win->nx * win->tile_size[0]);
  wp.win_hi[1] = (float)(win->ny * win->tile_size[1]);
  wp.win_hi[2] = (float)win->tile_size[2];
  for (int a = 0; a < 3; ++a) {
    wp.scene_lo[a] = (float)(win->scene_lo[a] - win->origin[a]);
    wp.scene_hi[a] = (float)(win->scene_hi[a] - win->origin[a]);
    wp.inv_size[a] = (float)(1.0 / win->tile_size[a]);
  }
  wp.split[0] = (float)win->tile_size[0];
  wp.split[1] = (float)win->tile_size[1];
  wp.nx = win->nx;
  wp.ny = win->ny;
  for (int q = 0; q < 4; ++q) wp.slot[q] = q < n_slots ? win->slot[q] : 0;
  wp.n_slots = n_slots;
  SamplerParams sp;
  sp.K_ray = sampler->K_ray;
  sp.K_min = sampler->K_min;
  sp.K_max = sampler->K_max;
  sp.render = sampler->render ? 1 : 0;
  sp.seed = sampler->seed;
  sp.iteration = sampler->iteration;
  sp.use_state_iteration = 0;
  sp.occ_res = 0;
  sp.occ = nullptr;
  if (sampler->mode < SNK_SAMPLE_SEGMENTS || sampler->mode > SNK_SAMPLE_POINTS ||
      (sampler->mode == SNK_SAMPLE_POINTS && sampler->K_min < 2))
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: bad sampler mode");
  sp.mode = sampler->mode;

  std::lock_guard<std::mutex> lock(g_mutex);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(err, err_len, SNK_ERR_CUDA, "snk_sample_segments_static: no current CUDA device");
  }
  if (g_scratch_dev[dev] == nullptr) {
    // one-time set-up on this device (it is current): the scratch's device address
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return fail(err, err_len, SNK_ERR_CUDA, "snk_sample_segments_static: cudaGetSymbolAddress failed");
    }
    g_scratch_dev[dev] = static_cast<unsigned char *>(p);
  }
  unsigned char *base = g_scratch_dev[dev];
  DevView *views = reinterpret_cast<DevView *>(base);
  if (B > 0 && scan_blocks(B) > kStaticMaxScanBlocks)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "snk_sample_segments_static: batch exceeds the scan scratch");

  for (int v = 0; v < n_views; ++v) {
    const snk_camera &c = cams[v];
    DevView &d = g_views_host[v];
    memset(&d, 0, sizeof(d));
    d.kind = c.kind;
    d.width = c.width;
    d.height = c.height;
    d.crop_r0 = c.crop_r0;
    d.crop_c0 = c.crop_c0;
    d.crop_h = c.crop_h;
    d.crop_w = c.crop_w;
    memcpy(d.a, c.a, sizeof(d.a));
    memcpy(d.b, c.b, sizeof(d.b));
    memcpy(d.off, c.off, sizeof(d.off));
    memcpy(d.scale, c.scale, sizeof(d.scale));
    memcpy(d.coef, c.coef, sizeof(d.coef));
    d.crop = nullptr;
  }
  // pageable source: the copy is staged before cudaMemcpyAsync returns, so the host staging can be reused
  if (cudaMemcpyAsync(views, g_views_host, sizeof(DevView) * n_views, cudaMemcpyHostToDevice,
                      (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(err, err_len, SNK_ERR_CUDA, "snk_sample_segments_static: camera copy failed");
  }
  RayBuffers rb{};
  rb.ray_od = ray_od;
  rb.ray_ok = ray_ok;
  rb.seg_slot = seg_slot;
  rb.seg_t = seg_t;
  rb.seg_n = seg_n;
  rb.seg_off = seg_off;
  rb.cnt = reinterpret_cast<uint32_t *>(base + kViewsBytes);
  rb.excl = reinterpret_cast<uint32_t *>(base + kViewsBytes + kRowsBytes);
  rb.block_tot = reinterpret_cast<uint32_t *>(base + kViewsBytes + 2 * kRowsBytes);
  rb.smp_t = smp_t;
  rb.smp_dt = smp_dt;
  rb.smp_xyz = smp_xyz;
  const cudaError_t e = launch_sample_segments(views, n_views, wp, sp, pix, B, 0, rb, cap, state, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(err, err_len, SNK_ERR_CUDA, cudaGetErrorString(e));
  return SNK_OK;
}
