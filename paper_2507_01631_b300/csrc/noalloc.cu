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

// The caller's message buffer (nullable), prefixed with this entry point's name.
int fail(char *err, int err_len, int code, const char *msg) {
  if (err && err_len > 0) snprintf(err, (size_t)err_len, "snk_sample_segments_static: %s", msg);
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
  char msg[256] = {0};
  const ErrSink sink{msg, sizeof(msg)};
  if (B < 0 || B > kStaticMaxRays)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "B must be in 0..65536 (the fixed scratch holds 65536 rays)");
  if (!cams || n_views < 1 || n_views > kMaxViews)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "NULL cameras or not 1..256 views");
  if (B > 0 && (!pix || !ray_od || !ray_ok || !seg_slot || !seg_t || !seg_n || !seg_off || !smp_t || !smp_dt ||
                !smp_xyz || !state))
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "NULL buffer");
  // the same descriptor checks and binary32 constants as snk_sample_segments
  WinParams wp;
  if (!win) return fail(err, err_len, SNK_ERR_INVALID_ARG, "window is NULL");
  if (check_window(sink, win, win->nx * win->ny, &wp) != SNK_OK) return fail(err, err_len, SNK_ERR_INVALID_ARG, msg);
  SamplerParams sp;
  if (check_sampler(sink, sampler, &sp) != SNK_OK) return fail(err, err_len, SNK_ERR_INVALID_ARG, msg);
  if (sp.occ_res != 0)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "no occupancy culling (its per-segment counts have no scratch here)");
  for (int v = 0; v < n_views; ++v) {
    DevView tmp;
    if (check_camera(sink, cams[v], v, &tmp) != SNK_OK) return fail(err, err_len, SNK_ERR_INVALID_ARG, msg);
  }
  // The camera copy below reads one static host staging array: a captured copy would replay
  // whatever the latest call left there, so calls on a capturing stream are refused.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "the stream's capture status could not be read");
  }
  if (cs != cudaStreamCaptureStatusNone)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "the stream is capturing a graph: calls cannot be captured");

  std::lock_guard<std::mutex> lock(g_mutex);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(err, err_len, SNK_ERR_CUDA, "no current CUDA device");
  }
  if (g_scratch_dev[dev] == nullptr) {
    // one-time set-up on this device (it is current): the scratch's device address
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return fail(err, err_len, SNK_ERR_CUDA, "cudaGetSymbolAddress failed");
    }
    g_scratch_dev[dev] = static_cast<unsigned char *>(p);
  }
  unsigned char *base = g_scratch_dev[dev];
  DevView *views = reinterpret_cast<DevView *>(base);
  if (B > 0 && scan_blocks(B) > kStaticMaxScanBlocks)
    return fail(err, err_len, SNK_ERR_INVALID_ARG, "batch exceeds the scan scratch");

  for (int v = 0; v < n_views; ++v) check_camera(sink, cams[v], v, &g_views_host[v]);  // checked above
  // pageable source: the copy is staged before cudaMemcpyAsync returns, so the host staging can be reused
  if (cudaMemcpyAsync(views, g_views_host, sizeof(DevView) * n_views, cudaMemcpyHostToDevice,
                      (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(err, err_len, SNK_ERR_CUDA, "camera copy failed");
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
