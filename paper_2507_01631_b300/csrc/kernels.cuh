// Internal interfaces between the translation units of libsnk.
#pragma once
#include <atomic>

#include "common.cuh"

namespace snk {

// Launch shapes picked by snk_autotune (defaults: the measured best on the 2x2 window).
struct Tuning {
  int tc_fwd_ctas = 3;          // tensor-core forward: persistent CTAs per SM (1, 2, 3)
  int tc_fwd_levels = 1;        // tensor-core forward: levels whose corner loads are issued together (1, 2)
  int tc_fwd_split = 1;         // tensor-core forward: dedicated gather warps, 2 CTAs per SM (0, 1)
  int tc_bwd_saved = 1;         // tensor-core training step: the forward stores activations for the backward (0, 1)
  int fp32_ctas = 2;            // binary32 field kernels: persistent CTAs per SM (1, 2)
  int composite_threads = 256;  // compositing: threads per block (64 .. 512, multiple of 32)
  int sampler_threads = 256;    // ray and sample kernels: threads per block (128 .. 512, multiple of 32)
};

// Adds n to the library-wide count of launched kernels (snk_launch_count).
void count_launches(int n);

// Where a failing check writes its message (a context's error text, or a caller's buffer;
// buf may be null): operator() formats the message and returns `code`.
struct ErrSink {
  char *buf;
  size_t len;
  int operator()(int code, const char *fmt, ...) const;
};
// Descriptor checks shared by every entry point that takes the descriptor (checks.cu):
// SNK_OK with the kernel constants in *o, else SNK_ERR_INVALID_ARG and a message.
int check_window(const ErrSink &fail, const snk_window *w, int n_slots, WinParams *o);
int check_sampler(const ErrSink &fail, const snk_sampler *s, SamplerParams *o);
// Camera v of a view list: kind, crop range, non-zero RPC normalisation scales; *d gets the
// kernels' copy (crop pointer null).
int check_camera(const ErrSink &fail, const snk_camera &c, int v, DevView *d);

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current device, once per
// device (the attribute belongs to that device's context; `done` is the caller's per-kernel
// mask of devices already set, devices >= 32 are set on every call).
template <typename K>
cudaError_t set_smem_limit(K kernel, int bytes, std::atomic<uint32_t> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint32_t bit = dev >= 0 && dev < 32 ? 1u << dev : 0u;
  if (bit != 0u && (done.load(std::memory_order_acquire) & bit) != 0u) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Workspace of one ray batch (context-owned, or caller buffers for the stage API).
struct RayBuffers {
  float *ray_od;       // [6][B]
  uint8_t *ray_ok;     // [B]
  uint8_t *seg_slot;   // [B][3]
  float *seg_t;        // [B][3][2]
  uint32_t *seg_n;     // [B][3]
  uint32_t *seg_off;   // [B][3]
  uint32_t *seg_k;     // [B][3] stratified candidates per segment (occupancy culling), or null
  uint32_t *cnt;       // [5][B]  per-slot sample counts, row 4 = accepted flag
  uint32_t *excl;      // [5][B]  exclusive scans of cnt within a scan block
  uint32_t *block_tot; // [5][nb] scan block totals, then bases
  float *smp_t;        // [cap]
  float *smp_dt;       // [cap]
  float *smp_xyz;      // [cap][3]
  uint32_t *smp_ray;   // [cap] ray of each sample (the view-direction colour input), or null
};

int scan_blocks(int B);
cudaError_t launch_sample_segments(const DevView *views, int n_views, const WinParams &win, const SamplerParams &smp,
                                   const uint32_t *pix, int B, int need_targets, const RayBuffers &rb, int64_t cap,
                                   snk_state *state, cudaStream_t st, const Tuning &tu = Tuning());

// Everything a field kernel needs to know about a model.
struct ModelDev {
  GridParams grid;
  int32_t in_dim, geo_out, colour, shared_colour, n_slots, mixed;
  int32_t e4m3;  // mixed path with an E4M3 first-layer input (one scale per slot and step)
  int32_t view_dirs, col_in;  // colour input [g | SH_16(direction)] and its width (geo_out + 16 view_dirs)
  int64_t tile_params, grid_params, colour_params, colour_base;
  int64_t w1, w2, w3;  // offsets of the density-MLP matrices inside a slot block
  int64_t v1, v2, v3;  // offsets of the colour-MLP matrices inside a colour block
};

enum FieldMode { kEncodeOnly = 0, kForward = 1, kBackward = 2 };

struct FieldArgs {
  ModelDev m;
  const float *params;        // binary32 master weights
  const uint16_t *params_lp;  // FP16 working copy of tables and MLP weights (mixed)
  float *grads;
  const float *xyz;           // [S][3] tile-local sample positions
  const float *feat_in;       // [S][IN] features instead of encoding (MLP-only API), or null
  float *feat_out;            // [S][IN] encoded features (encode API), or null
  uint32_t *idx_out;          // [S][L][8] corner entries (encode API), or null
  float *sigma_rgb;           // forward output [S][4]
  const float *dsr;           // backward input [S][4]
  float *dfeat_out;           // backward: write dfeat here instead of scattering, or null
  uint16_t *feat_lp;          // mixed path: FP16 features per 128-sample tile (forward writes, backward reads)
  float *feat32;              // E4M3 path: [S][IN] binary32 features (gather writes, forward reads)
  uint8_t *codes;             // E4M3 path: [S][IN] first-layer codes (forward writes, backward reads)
  uint32_t *amax;             // E4M3 path: per slot, bits of max |feature| of the step (>= 0 floats)
  uint16_t *acts;             // tensor-core training step: stored activations, act_tile_bytes a tile, or null
  const uint16_t *cells_lp;   // mixed forward: cell-major FP16 copy of the dense levels ([n_slots][n_cells][8] pairs), or null
  float *cell_grad;           // mixed backward: cell-major binary32 gradients of the dense levels ([n_slots][n_cells][8]
                              // pairs; zero between steps), or null (dense levels then add into grads directly)
  const uint32_t *smp_ray;    // view-direction models: [S] ray of each sample
  const float *ray_od;        // view-direction models: [6][n_rays] ray origins and directions
  int32_t n_rays;
  const snk_state *state;
  int64_t S;                  // extent of the slot-major arrays
  int32_t slot_only;          // -1: every slot; k: only slot k (per-tile launches)
  int32_t mode;
};
cudaError_t launch_field_fp32(const FieldArgs &a, int sm_count, cudaStream_t st, const Tuning &tu = Tuning());
cudaError_t launch_field_tc(const FieldArgs &a, int sm_count, cudaStream_t st, const Tuning &tu = Tuning());
// One CTA in a bounded mbarrier wait that completes (arrive != 0) or gives up (timeout bit).
cudaError_t launch_wait_selftest(int arrive, snk_state *state, cudaStream_t st);
// Bytes of one 128-sample tile of stored activations (FieldArgs::acts).
int64_t act_tile_bytes(bool colour, bool view_dirs);
// Scatter-add feat_in (read as dfeat [S][L*F]) into the table gradients.
cudaError_t launch_encode_scatter(const FieldArgs &a, cudaStream_t st);
// E4M3 path, first pass: binary32 features from the FP16 tables into feat32 and
// the per-slot max |feature| into amax (which must be zero before the launch).
cudaError_t launch_gather_amax(const FieldArgs &a, int sm_count, cudaStream_t st);
// Crops and ray pool of a window (crops.cu).
struct CropParams {
  double tile[2];  // tile extent in x, y (metres)
  int32_t margin;  // pixels added on every side of a tile's corner box
};
cudaError_t launch_crops(const DevView *views, int n_views, const WinParams &win, const CropParams &cp,
                         int32_t *tile_rects, int32_t *view_rects, cudaStream_t st);
int64_t pool_chunks(int64_t max_pixels);
// n_pool[0] = pool entries written (<= cap), n_pool[1] = accepted pixels in all crops
cudaError_t launch_ray_pool(const DevView *views, int n_views, const WinParams &win, const int32_t *view_rects,
                            int64_t *base, int64_t max_pixels, uint8_t *flags, uint32_t *chunk_cnt, uint32_t *pool,
                            int64_t cap, uint32_t *n_pool, cudaStream_t st);
cudaError_t launch_draw(const uint32_t *pool, const uint32_t *n_pool, int B, uint32_t seed, uint32_t iteration,
                        uint32_t *pix, cudaStream_t st);
// Occupancy grid update (occupancy.cu).
cudaError_t launch_occ_points(int n_slots, int R, uint32_t seed, uint32_t step, float *xyz, uint32_t *ray,
                              snk_state *state, cudaStream_t st);
int64_t occ_partials(int n_slots, int R);
cudaError_t launch_occ_update(int n_slots, int R, const float *sigma_rgb, float decay, float threshold,
                              float *density, uint8_t *occ, float *partial, float *thr, cudaStream_t st);
// codes[i] = E4M3(x[i] / scale), the conversion the E4M3 path uses.
cudaError_t launch_quantize_e4m3(const float *x, int64_t n, float scale, uint8_t *codes, cudaStream_t st);

struct CompositeArgs {
  const float *sigma_rgb;
  const float *smp_t;
  const float *smp_dt;
  const uint32_t *seg_n;
  const uint32_t *seg_off;
  int32_t B;
  float *out;             // [B][5] or null
  float *t_final;         // [B] or null
  const float *g_rgb;     // [B][3] upstream gradient (stage API), or null
  const uint32_t *pix;    // training: pixels for the targets
  const DevView *views;
  float *dsr;             // [S][4] backward output, or null (forward only)
  snk_state *state;
  int32_t train;          // 1: MSE loss against targets, gradient scaled by the loss scale
};
cudaError_t launch_composite(const CompositeArgs &a, cudaStream_t st, const Tuning &tu = Tuning());

struct AdamArgs {
  float *params;
  uint16_t *params_lp;
  float *grads;
  float *m;
  float *v;
  int32_t *steps;
  int64_t n;
  int32_t n_groups;
  int64_t start[9], end[9], mlp_start[9];
  float lr, beta1, beta2, eps, l2;
  snk_state *state;
  int32_t mixed;
  uint32_t bwd_mode;  // written to state->bwd_mode: 0 binary32, 1 stored activations, 2 recomputed
};
cudaError_t launch_adam(const AdamArgs &a, int sm_count, cudaStream_t st);
// Diagnostic (probe.cu): n_ops reductions of `width` (8 or 16) bytes of 1.0f to random
// 16-byte slots of table [n16][4] floats.
cudaError_t launch_red_probe(float *table, int64_t n16, int64_t n_ops, int width, uint32_t seed, int sm_count,
                             cudaStream_t st);
// Cell-major copies of the dense levels (cells.cu): the FP16 corner pairs of every cell of every
// slot's dense levels from the working copy; and the fold of the cell-major gradients into the
// table gradients (each vertex sums the corners it is of its up to 8 cells), clearing them.
cudaError_t launch_cells_copy(const uint16_t *params_lp, int64_t tile_params, const GridParams &gp, int n_slots,
                              uint16_t *cells, int sm_count, cudaStream_t st);
cudaError_t launch_cells_fold(float *cell_grad, float *grads, int64_t tile_params, const GridParams &gp, int n_slots,
                              int sm_count, cudaStream_t st);
// lp[i] = FP16(w[i]) (round to nearest even) for i < n: the mixed model's working copy.
cudaError_t launch_refresh_lp(const float *w, uint16_t *lp, int64_t n, int sm_count, cudaStream_t st);

}  // namespace snk
