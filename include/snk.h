/*
 * snk.h - C ABI of libsnk, the B300 (sm_103a) training step of a Snake-NeRF
 * tile or 2x2 tile window ("Tile and Slide", Billouard et al., ICCV 2025).
 *
 * One step: rays from satellite cameras (Sec. 3, Sec. 4.6 "On-the-fly Ray
 * Calculation") -> window acceptance and segmented sampling (Sec. 4.4, 4.5)
 * -> multiresolution hash encoding per tile (Sec. 4.1, NGP) -> local density
 * MLP and shared colour MLP (Sec. 4.1) -> volume rendering (NeRF Eq. 3,
 * Sec. 4.5) -> colour loss, backward and Adam (Sec. 4.4, 4.6).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status (SNK_OK = 0 or an SNK_ERR_* code);
 *    snk_last_error() gives a message for the last failing call on a context.
 *    Invalid arguments are reported before anything is launched.
 *  - Data pointers are DEVICE pointers owned by the caller unless a
 *    parameter says "host".  The library never frees caller memory.  The
 *    context owns only its workspace (snk_ctx_reserve) and its copy of the
 *    views (snk_set_views); snk_ctx_destroy frees both.
 *  - A context belongs to the device given to snk_ctx_create.  Every other
 *    call on it runs on the calling thread's current device, which must be
 *    that device (and the stream one of its streams); snk_ctx_create and
 *    snk_ctx_destroy make it current themselves.  Contexts on different
 *    devices may live in one process.
 *  - Calls are asynchronous on the given stream (NULL = legacy default
 *    stream) unless they return a host value.  A call that needs more
 *    workspace than reserved grows it with cudaMalloc, which synchronises the
 *    device; reserve first to keep calls asynchronous and capturable.
 *  - Floating point is binary32 unless stated; the camera model is evaluated
 *    in binary64.  Discrete results (acceptance, segment bounds, sample
 *    counts and offsets, hash indices) follow a fixed sequence of IEEE
 *    operations and are reproducible bit for bit.
 *  - Sample arrays are SLOT-MAJOR: the samples of parameter slot k occupy
 *    [slot_base[k], slot_base[k] + slot_count[k]) and slot_base[k] is a
 *    multiple of 128.  Inside a slot, the samples of a ray segment are
 *    contiguous and ordered along the ray; segments appear in ray order.
 *    Padding entries between slots are never read as samples.
 *
 * Parameter layout (flat, per model):
 *    [slot 0 | ... | slot n-1 | colour block(s)]
 *    slot block   = hash table (n_entries x F, entry-major) | W1 | W2 | W3
 *    colour block = V1 | V2 | V3          (matrices row-major [out][in])
 *  with n_entries, offsets and sizes given by snk_model_layout().
 */
#ifndef SNK_H
#define SNK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *snk_stream_t; /* a cudaStream_t */
typedef struct snk_ctx snk_ctx;

enum {
    SNK_OK = 0,
    SNK_ERR_INVALID_ARG = 1,  /* bad descriptor, size or NULL pointer */
    SNK_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    SNK_ERR_OOM = 3,          /* workspace allocation failed */
    SNK_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
    SNK_ERR_DEVICE_CHECK = 5, /* a device-side bounds or capacity check fired */
    SNK_ERR_OVERFLOW = 6      /* non-finite gradients: Adam step skipped, loss scale halved */
};

/* Camera kinds (Sec. 4.3 names the RPC model; affine is its linear case). */
enum { SNK_CAM_AFFINE = 0, SNK_CAM_RPC3 = 1 };
/* Precision of a model.
 *  SNK_FP32:  binary32 tables, MLPs and gradients.
 *  SNK_MIXED: FP16 working copy of every parameter, MLPs on the tensor cores
 *             with FP32 accumulation, binary32 master weights, dynamic loss scale.
 *  SNK_MIXED_E4M3: SNK_MIXED with the density MLP's first-layer input (the
 *             encoded features) quantised to E4M3 (OCP FP8: 4 exponent bits,
 *             3 mantissa bits, largest 448; round to nearest even, saturating).
 *             One scale per slot and step, amax / 448 over the slot's features
 *             of the current batch; the layer sees scale x value(code).  The
 *             backward passes the feature gradient straight through the
 *             quantiser. */
enum { SNK_FP32 = 0, SNK_MIXED = 1, SNK_MIXED_E4M3 = 2 };

/* One view: its localisation map (r, c, h) -> (x, y) and its resident crop.
 *  AFFINE: x = a0 + a1 c + a2 r + a3 h, y = b0 + b1 c + b2 r + b3 h.
 *  RPC3:   with rn = (r - off[0]) / scale[0], cn = (c - off[1]) / scale[1],
 *          hn = (h - off[2]) / scale[2]:
 *          x = off[3] + scale[3] * Nx / Dx,  y = off[4] + scale[4] * Ny / Dy,
 *          Nx, Dx, Ny, Dy = coef[0..3] . m(cn, rn, hn), the 20 cubic monomials
 *          1, c, r, h, cr, ch, rh, c^2, r^2, h^2, crh, c^3, cr^2, ch^2, c^2 r,
 *          r^3, rh^2, c^2 h, r^2 h, h^3 (each a left-to-right product, the sum
 *          taken left to right).
 *  (r, c) are full-image pixel coordinates; pixel (row, col) is sampled at its
 *  centre (row + 0.5, col + 0.5).  The crop (crop_r0, crop_c0, crop_h, crop_w)
 *  is the part of the image whose target colours are resident (Sec. 4.3). */
typedef struct {
    int32_t kind;
    int32_t width, height;
    int32_t crop_r0, crop_c0, crop_h, crop_w;
    int32_t reserved;
    double a[4], b[4];
    double off[5], scale[5];
    double coef[4][20];
} snk_camera;

/* A window of nx x ny loaded tiles (nx, ny in {1, 2}) inside a scene box
 * (Sec. 4.2, 4.4).  Scene-metre boxes; all tiles share z_min = origin[2] and
 * height tile_size[2].  slot[iy * nx + ix] is the parameter slot of tile
 * (ix, iy), a permutation of 0..nx*ny-1. */
typedef struct {
    double origin[3];
    double tile_size[3];
    double scene_lo[3], scene_hi[3];
    int32_t nx, ny;
    int32_t slot[4];
} snk_window;

/* Model sizes.  Grid: L levels of F = 2 features, T = 2^log2_T entries,
 * resolutions n_min .. n_max (NGP).  Density MLP: L*F -> 64 -> 64 -> geo_out
 * (ReLU hidden, no biases).  geo_out = 4 without a colour net (rgb =
 * sigmoid(g1..3)); geo_out = 16 with a colour MLP 16 -> 64 -> 64 -> 3,
 * shared by all slots (shared_colour = 1, the paper's global colour network)
 * or one per slot.  Supported: L*F in {8, 16, 32}, hidden = 64, n_slots 1..4. */
typedef struct {
    int32_t L, F, log2_T, n_min, n_max;
    int32_t hidden;
    int32_t geo_out;
    int32_t colour;
    int32_t shared_colour;
    int32_t n_slots;
    int32_t precision; /* SNK_FP32, SNK_MIXED or SNK_MIXED_E4M3 */
    int32_t view_dirs; /* 1: the colour MLP's input is [embedding | 16 real spherical harmonics of
                        * degrees 0..3 of the ray's unit direction] (the view-direction variant,
                        * after Instant-NGP's direction encoding); V1 is then [64][geo_out + 16].
                        * Needs a colour MLP; used by snk_train_step and snk_render (the stage
                        * calls have no ray directions and reject it) */
} snk_model;

/* Layout facts computed from a model on the host (no GPU needed). */
typedef struct {
    int32_t res[32];           /* N_l */
    int32_t dense[32];         /* 1 if (N_l + 1)^3 <= T */
    int64_t level_offset[32];  /* first entry of level l */
    int64_t level_size[32];    /* entries of level l (multiple of 8) */
    int64_t n_entries;         /* entries per table */
    int64_t grid_params;       /* n_entries * F */
    int64_t tile_params;       /* one slot block */
    int64_t colour_params;     /* one colour block */
    int64_t n_params;          /* whole flat vector */
    int32_t n_optimisers;      /* slots + colour blocks */
    int32_t n_colour_blocks;
} snk_layout;

/* Sampler modes.
 *  SNK_SAMPLE_SEGMENTS (the paper's segmented sampler, Sec. 4.5): each segment
 *    of a ray gets K = clamp(rint(K_ray len_seg / len_ray), K_min, K_max) bins
 *    of width w = len_seg / K and a sample at t0 + (k + u) w, delta = w.
 *  SNK_SAMPLE_UNIFORM (the NeRF-XL distribution the paper compares against):
 *    K_ray bins over the ray's whole scene interval, sample j at
 *    t_in + (j + u) w; each sample belongs to the tile holding its point and
 *    the samples of a tile form its segment (seg_t = the ray's [t_in, t_out]);
 *    delta = w.
 *  SNK_SAMPLE_POINTS (point samples, the variant of the paper's remark on the
 *    face point): K points per segment at t0 + k (len_seg / (K - 1)), the last
 *    exactly at t1, and delta_i = t_i - t_{i-1} along the ray (0 for the
 *    ray's first point): the face point of two segments is sampled twice and
 *    the second copy has delta 0.  Needs K_min >= 2; no jitter. */
enum { SNK_SAMPLE_SEGMENTS = 0, SNK_SAMPLE_UNIFORM = 1, SNK_SAMPLE_POINTS = 2 };

/* Sampler: samples per segment K = clamp(rint(K_ray len_seg / len_ray),
 * K_min, K_max); render = 1 puts every sample at its bin centre.
 * Occupancy culling (Sec. 4.1, SAT-NGP's coarse voxel grid): with occ_res > 0
 * the K stratified candidates of a segment are placed as without culling and
 * only those whose cell of the slot's grid is occupied become samples (each
 * keeps its bin width as delta); seg_n then counts the kept samples.  The grid
 * of slot k is occupancy[k * R^3 ...], cell (x, y, z) = min(floor(l R), R - 1)
 * of the tile-local position l (binary32), stored at (z R + y) R + x; nonzero =
 * occupied.  snk_occupancy_update maintains such a grid. */
typedef struct {
    int32_t K_ray, K_min, K_max;
    int32_t render;
    uint32_t seed;
    uint32_t iteration;       /* Philox key word; the training step uses its own counter */
    int32_t occ_res;          /* cells per axis of each slot's occupancy grid; 0: no culling */
    int32_t mode;             /* SNK_SAMPLE_SEGMENTS (default), _UNIFORM or _POINTS; culling needs _SEGMENTS */
    const uint8_t *occupancy; /* device [n_slots][occ_res^3], or NULL when occ_res = 0 */
} snk_sampler;

/* Adam hyper-parameters (I-NGP's: 1e-2, 0.9, 0.99, 1e-15, 1e-6). */
typedef struct {
    float lr, beta1, beta2, eps, l2_mlp;
} snk_adam;

/* Trainable state, all device memory of n_params entries (snk_layout). */
typedef struct {
    float *params;       /* binary32 master weights */
    uint16_t *params_lp; /* SNK_MIXED*: FP16 working copy of all parameters (tables and MLP weights); else NULL */
    float *grads;        /* gradient accumulator; must be zero before a step, zeroed by the step */
    float *adam_m;
    float *adam_v;
    int32_t *adam_step;  /* n_optimisers step counts (device), incremented by each step */
} snk_params;

/* Per-step device state (caller-owned device memory, zero-initialise once,
 * then set loss_scale; the step updates it). */
typedef struct {
    float loss;          /* MSE of the last step */
    float loss_scale;    /* dynamic loss scale (SNK_MIXED); 1 for SNK_FP32 */
    uint32_t n_accepted; /* accepted rays of the last step */
    uint32_t n_samples;  /* samples of the last step */
    uint32_t status;     /* bit 0: overflow skip, bit 1: device check, bit 2: timeout */
    int32_t good_steps;  /* consecutive finite steps (loss-scale growth) */
    uint32_t iteration;  /* step counter, Philox key word of the stratified jitter */
    uint32_t slot_base[5];
    uint32_t slot_count[4];
    uint32_t nonfinite;  /* internal: set during a step whose gradients are not all finite */
    uint32_t bwd_mode;   /* backward of the last training step: 0 binary32 path, 1 the tensor-core
                          * backward read the activations its forward stored, 2 it recomputed them
                          * (the stored-activation buffer exceeded the context's activation budget
                          * or could not be allocated, or tc_bwd_saved = 0) */
    uint32_t reserved;
} snk_state;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device` (made current).  *out is NULL on error. */
int snk_ctx_create(int device, snk_ctx **out);
/* Free the context and its workspace (synchronises the device).  NULL is a no-op. */
int snk_ctx_destroy(snk_ctx *ctx);
/* Size the workspace for batches of up to max_rays rays and max_samples samples. */
int snk_ctx_reserve(snk_ctx *ctx, int64_t max_rays, int64_t max_samples);
/* Most device memory (bytes) the context may hold for stored activations (the
 * tensor-core training step's per-sample activations, 544 B a sample of sample
 * capacity with a colour network).  A training step whose capacity needs more
 * -- or whose buffer cudaMalloc cannot provide -- does not fail: it runs the
 * backward that recomputes the forward's activations instead (the per-sample
 * activations are recomputed instead of stored when batches outgrow memory;
 * same results up to the order of float atomics), and writes 2 into
 * snk_state.bwd_mode.  bytes < 0: no budget (the default; only cudaMalloc
 * limits it).  A budget below the buffer the context already holds frees that
 * buffer (synchronising the device). */
int snk_ctx_set_act_budget(snk_ctx *ctx, int64_t bytes);
/* Host only: the sample capacity a step of B rays with this window and sampler
 * sizes its workspace for (an upper bound of the batch's samples, Sec. 4.5:
 * K_ray a ray in uniform mode, else at most max(s K_min, (s - 1) K_min + K_ray)
 * + s and at most s K_max for a window whose rays have up to s segments, plus
 * slot alignment), so that snk_ctx_reserve(ctx, B, snk_max_samples(...)) sizes
 * the context once before graph capture.  Returns -1 for a NULL argument. */
int64_t snk_max_samples(const snk_window *win, const snk_sampler *sampler, int64_t B);
/* Message of the last failing call on ctx (static storage of the context). */
const char *snk_last_error(const snk_ctx *ctx);
/* Library version string (host, static). */
const char *snk_version(void);
/* Host only: sizeof of the ABI structs, in the order snk_camera, snk_window,
 * snk_model, snk_layout, snk_sampler, snk_adam, snk_params, snk_state,
 * snk_tuning, written to sizes[0..n-1] (n <= 9).  Lets a binding check its struct mirrors.  Returns
 * the number written. */
int snk_abi_sizes(int64_t *sizes, int n);

/* Host only: grid level resolutions/offsets and parameter counts (NGP, Sec. 4.1).
 * Returns SNK_ERR_INVALID_ARG for unsupported sizes.  Needs no GPU. */
int snk_model_layout(const snk_model *model, snk_layout *out);

/* Copy n_views cameras (host array) and per-view crop pointers (host array of
 * device pointers to crop_h x crop_w x 3 binary32 images, or NULL when no
 * targets are needed) into the context.  Set-up call: it synchronises
 * `stream`, so the host arrays may be reused after it returns.  At most 256
 * views.  Sec. 4.3 (crops), Sec. 4.6 (rays from the cameras). */
int snk_set_views(snk_ctx *ctx, const snk_camera *cams, int n_views, const float *const *crops,
                  snk_stream_t stream);

/* FP16 working copy of a mixed-precision model's parameters: p->params_lp[i] =
 * the binary32 p->params[i] rounded to the nearest FP16 (ties to even), for all
 * n_params entries (snk_layout), on `stream`.  C12's working copy: a mixed
 * model's first step needs it written once from the initial master weights
 * (every training step refreshes it after Adam).  SNK_ERR_INVALID_ARG for a
 * binary32 model or a NULL params / params_lp. */
int snk_params_refresh_lp(snk_ctx *ctx, const snk_model *model, const snk_params *p, snk_stream_t stream);

/* ---- stages ----------------------------------------------------------- */

/* Rays, acceptance, segments and stratified samples for B packed pixel ids
 * pix[i] = view << 24 | row << 12 | col (Sec. 4.4, 4.5, 4.6).
 * Outputs (device, caller-allocated):
 *   ray_od    [6][B]   o.x, o.y, o.z, d.x, d.y, d.z (window-local metres, unit d)
 *   ray_ok    [B]      1 if accepted
 *   seg_slot  [B][3]   slot of each segment, 255 if unused
 *   seg_t     [B][3][2] t0, t1 of each segment
 *   seg_n     [B][3]   samples per segment (0 if unused)
 *   seg_off   [B][3]   first sample of each segment in the slot-major arrays
 *   smp_t, smp_dt [cap], smp_xyz [cap][3] (tile-local [0,1]^3)
 *   state     device snk_state: n_accepted, n_samples, slot_base, slot_count
 * cap = capacity of the sample arrays; if the slot-major extent exceeds it,
 * no sample is written and status bit 1 is set (SNK_ERR_DEVICE_CHECK from
 * snk_sync_status).  A pixel whose view does not exist is rejected with the
 * same status bit.  Jitter: Philox-4x32-10 (Salmon et al. 2011), key
 * (seed, iteration), counter (ray, j >> 2, 1, 0), lane j & 3, j = index of
 * the sample along its ray. */
int snk_sample_segments(snk_ctx *ctx, const snk_window *win, const uint32_t *pix, int B,
                        const snk_sampler *sampler, float *ray_od, uint8_t *ray_ok, uint8_t *seg_slot,
                        float *seg_t, uint32_t *seg_n, uint32_t *seg_off, float *smp_t, float *smp_dt,
                        float *smp_xyz, int64_t cap, snk_state *state, snk_stream_t stream);

/* Hash encoding (Sec. 4.1, NGP) of S slot-major samples: feat [S][L*F]
 * binary32, level-major.  Samples outside the slot ranges of `state` are
 * skipped.  idx_out (nullable) [S][L][8] receives the table entry index of
 * each corner (within the slot's table) for bit-exact checks. */
int snk_encode(snk_ctx *ctx, const snk_model *model, const snk_params *p, const float *smp_xyz,
               const snk_state *state, int64_t S, float *feat, uint32_t *idx_out, snk_stream_t stream);
/* Adds dfeat [S][L*F] scattered with the trilinear weights into p->grads (tables). */
int snk_encode_backward(snk_ctx *ctx, const snk_model *model, const snk_params *p, const float *smp_xyz,
                        const snk_state *state, int64_t S, const float *dfeat, snk_stream_t stream);

/* Density + colour MLPs (Sec. 4.1) on features feat [S][L*F]:
 * out [S][4] = (sigma, r, g, b). */
int snk_mlp(snk_ctx *ctx, const snk_model *model, const snk_params *p, const float *feat,
            const snk_state *state, int64_t S, float *out, snk_stream_t stream);
/* Backward of snk_mlp for upstream dout [S][4] = (dsigma, dr, dg, db): adds the
 * weight gradients into p->grads and writes dfeat [S][L*F]. */
int snk_mlp_backward(snk_ctx *ctx, const snk_model *model, const snk_params *p, const float *feat,
                     const snk_state *state, int64_t S, const float *dout, float *dfeat, snk_stream_t stream);

/* Volume rendering (NeRF Eq. 3, Sec. 4.5) of B rays from slot-major samples
 * (sigma_rgb [S][4], smp_t, smp_dt) reached through seg_n / seg_off:
 * out [B][5] = (r, g, b, depth, opacity), t_final [B] (nullable). */
int snk_composite(snk_ctx *ctx, const float *sigma_rgb, const float *smp_t, const float *smp_dt,
                  const uint32_t *seg_n, const uint32_t *seg_off, int B, float *out, float *t_final,
                  snk_stream_t stream);
/* Backward of snk_composite for per-ray colour gradients g_rgb [B][3]:
 * d_sigma_rgb [S][4] = (dsigma, dr, dg, db) for every sample of the rays. */
int snk_composite_backward(snk_ctx *ctx, const float *sigma_rgb, const float *smp_t, const float *smp_dt,
                           const uint32_t *seg_n, const uint32_t *seg_off, int B, const float *g_rgb,
                           float *d_sigma_rgb, snk_stream_t stream);

/* ---- whole step --------------------------------------------------------- */

/* One training step on B packed pixels (Sec. 4.4, last paragraph): rays,
 * segments, samples (jitter key = (sampler->seed, state->iteration)), encode,
 * MLPs, rendering, MSE loss over accepted rays against the views' crops,
 * backward, Adam per optimiser (slot tables + density MLP; colour net), then
 * state->iteration += 1.  SNK_MIXED adds dynamic loss scaling: a step with
 * non-finite gradients is skipped (status bit 0) and the scale halved.
 * Optional outputs (nullable): out [B][5] rendered (r, g, b, depth, opacity).
 * Never synchronises; read state (device) for loss and counts -- except when the
 * context's workspace must grow: the batch needs snk_max_samples(win, sampler, B)
 * samples of capacity and, on the tensor-core path with tc_bwd_saved (the
 * default), a stored-activation buffer for that capacity; the first step that
 * needs more allocates it (synchronising), so reserve before capturing a graph
 * and run one step eagerly.  SNK_ERR_OOM when the sample workspace cannot be
 * allocated; a stored-activation buffer that exceeds the activation budget
 * (snk_ctx_set_act_budget) or cannot be allocated is not an error: the step
 * recomputes the activations in its backward (state->bwd_mode = 2). */
int snk_train_step(snk_ctx *ctx, const snk_model *model, const snk_window *win, const uint32_t *pix, int B,
                   const snk_sampler *sampler, const snk_adam *adam, const snk_params *p, snk_state *state,
                   float *out, snk_stream_t stream);

/* Render B packed pixels (forward only, bin-centre samples): out [B][5]. */
int snk_render(snk_ctx *ctx, const snk_model *model, const snk_window *win, const uint32_t *pix, int B,
               const snk_sampler *sampler, const snk_params *p, snk_state *state, float *out,
               snk_stream_t stream);

/* E4M3 quantiser of the SNK_MIXED_E4M3 first layer: codes[i] = E4M3(x[i] /
 * scale) for n binary32 device values (the division rounded to nearest, then
 * rounded to nearest even on the E4M3 grid, magnitudes beyond 448 saturating).
 * Device buffers owned by the caller; scale must be positive and finite, else
 * SNK_ERR_INVALID_ARG.  The same conversion the training step applies with the
 * per-slot scale amax / 448. */
int snk_quantize_e4m3(snk_ctx *ctx, const float *x, int64_t n, float scale, uint8_t *codes, snk_stream_t stream);

/* Allocation-free variant of snk_sample_segments (the paper has no counterpart:
 * this exists for embedding).  For callers that cannot allocate device memory --
 * hosts whose own allocator owns all device memory, fixed-budget or real-time
 * runtimes, contexts where cudaMalloc would synchronise or is not allowed --
 * and that therefore cannot create an snk_ctx.  The caller passes the cameras
 * (host array, up to 256) and every input and output buffer exactly as for
 * snk_sample_segments, and gets the same results.  The library's scratch (the
 * cameras' device copy and the sample-count scans) lives in one fixed
 * file-scope device array of about 2.8 MB that every GPU which loads the
 * library holds until the process exits; nothing is allocated.
 *  - B may be at most 65536; larger batches return SNK_ERR_INVALID_ARG and a
 *    message in err (nullable, err_len bytes).  The window, sampler and
 *    cameras are checked exactly as snk_set_views and snk_sample_segments
 *    check them; occupancy culling is not offered (SNK_ERR_INVALID_ARG).
 *  - The first call on a device looks up the device address of the scratch on
 *    that device (the device current at the call).
 *  - Calls cannot be captured into a CUDA graph: every call copies the cameras
 *    from one static host staging array, which a replayed copy would read in
 *    whatever state the latest call left it.  A call on a stream that is
 *    capturing returns SNK_ERR_INVALID_ARG.  Calls queued on one stream
 *    without synchronising in between are fine: each call's copy consumes the
 *    staging array before the call returns.
 *  - Every call on a device shares the same scratch and leaves the last call's
 *    contents in it; nothing in it has to start at zero (each kernel writes what
 *    it later reads).  Calls that overlap on the GPU (other streams, other host
 *    threads) race on the scratch: serialise them.  Host threads are serialised
 *    by a lock around the set-up and the camera copy. */
int snk_sample_segments_static(const snk_window *win, const snk_camera *cams, int n_views, const uint32_t *pix,
                               int B, const snk_sampler *sampler, float *ray_od, uint8_t *ray_ok, uint8_t *seg_slot,
                               float *seg_t, uint32_t *seg_n, uint32_t *seg_off, float *smp_t, float *smp_dt,
                               float *smp_xyz, int64_t cap, snk_state *state, snk_stream_t stream, char *err,
                               int err_len);

/* ---- crops and ray pool of a window (Sec. 4.3, Sec. 4.4) ----------------- */

/* Image crops from ground tiles (Sec. 4.3): every view of the context
 * projects the 8 corners of each tile of the window (x, y of the tile's
 * corners, h = z_min and z_max) to continuous pixel coordinates and takes
 * rows [floor(min) - margin, ceil(max) + margin) and likewise columns,
 * clipped to the image (an empty rectangle if the tile is outside it).  The
 * projection solves localisation(row, col, h) = (x, y) by Newton's method in
 * binary64 (forward-difference Jacobian with one-pixel steps, 16 iterations
 * from the image centre).  Device outputs: tile_rects [n_views][4][4] =
 * (r0, c0, h, w) of window tile k = iy * nx + ix (zeros for k >= nx * ny),
 * view_rects [n_views][4] = the bounding rectangle of the view's non-empty
 * tile rectangles ((0, 0, 0, 0) if none). */
int snk_build_crops(snk_ctx *ctx, const snk_window *win, int margin, int32_t *tile_rects, int32_t *view_rects,
                    snk_stream_t stream);
/* Ray pool of the window: the packed pixels (view << 24 | row << 12 | col) of
 * every view's rectangle in view_rects (device, as written by
 * snk_build_crops) whose rays the window accepts (the acceptance of the
 * training step, Sec. 4.4), in (view, row, col) order, into pool (device, cap
 * entries).  n_pool (device, 2 x u32): [0] = entries written (<= cap), [1] =
 * accepted pixels in all crops (larger than [0] if cap was too small).  The
 * context keeps a scratch of one byte per image pixel of its views. */
int snk_ray_pool(snk_ctx *ctx, const snk_window *win, const int32_t *view_rects, uint32_t *pool, int64_t cap,
                 uint32_t *n_pool, snk_stream_t stream);
/* A batch of B pixels drawn uniformly from the pool (device pool, n_pool as
 * written by snk_ray_pool): pix[i] = pool[(x >> 8) * n_pool[0] >> 24], x =
 * word i % 4 of Philox-4x32-10 with counter (i / 4, 0, 0, 0) and key (seed,
 * iteration).  An empty pool gives pixels of no view, which a step rejects. */
int snk_draw_batch(snk_ctx *ctx, const uint32_t *pool, const uint32_t *n_pool, int B, uint32_t seed,
                   uint32_t iteration, uint32_t *pix, snk_stream_t stream);

/* ---- occupancy grid (Sec. 4.1, SAT-NGP's coarse voxel grid) -------------- */

/* Update the occupancy grids of all slots: every cell of slot k's R^3 grid
 * gets sigma at one point p = (cell + u) x (1 / R) (binary32 per axis; u = three
 * words of Philox-4x32-10 with counter (cell, k, 3, 0) and key (seed, step),
 * each (w >> 8) 2^-24), evaluated with the slot's field of `model` and `p` (the
 * kernels of a step, at the model's precision); then
 *   density <- max(decay x density, sigma)
 *   occupancy <- density > min(threshold, mean of slot k's density).
 * density [n_slots][R^3] binary32 and occupancy [n_slots][R^3] u8 are caller-
 * owned device arrays (cell (x, y, z) at (z R + y) R + x); start from density 0
 * and occupancy 1 everywhere (no culling before the first update).  R a
 * multiple of 8 in 8..512; uses the context's sample workspace for
 * n_slots R^3 samples (may grow it).  The grid feeds snk_sampler.occupancy. */
int snk_occupancy_update(snk_ctx *ctx, const snk_model *model, const snk_params *p, float *density,
                         uint8_t *occupancy, int R, float decay, float threshold, uint32_t seed, uint32_t step,
                         snk_stream_t stream);

/* ---- tile residency (snake sweep, Sec. 4.4) ------------------------------ */

/* Host only: bytes of one parked tile of `model`, a contiguous block laid out
 * (offsets rounded up to 256 bytes) as
 *   params (tile_params x f32) | adam_m (f32) | adam_v (f32) |
 *   params_lp (tile_params x u16; unused for SNK_FP32) | Adam step count (i32). */
int snk_tile_bytes(const snk_model *model, int64_t *bytes);
/* Copy the trainable state of parameter slot `slot` (its block of params,
 * params_lp, adam_m, adam_v and its step count) into dst, a block of
 * snk_tile_bytes bytes in pinned host memory or device memory (cudaMemcpyAsync
 * on `stream`, cudaMemcpyDefault: asynchronous for pinned or device memory).
 * The slot's gradients are not copied (they are zero between steps).  The slot
 * keeps its contents; the caller may then unpark another tile into it.
 * SNK_ERR_INVALID_ARG for a bad slot, model or NULL pointer. */
int snk_tile_park(snk_ctx *ctx, const snk_model *model, const snk_params *p, int slot, void *dst,
                  snk_stream_t stream);
/* Reverse of snk_tile_park: load a parked block into slot `slot`. */
int snk_tile_unpark(snk_ctx *ctx, const snk_model *model, const snk_params *p, int slot, const void *src,
                    snk_stream_t stream);

/* ---- launch shapes ------------------------------------------------------ */

/* Launch shapes of the context's kernels (the paper has no counterpart: they
 * change speed, never results beyond the order of float atomics). */
typedef struct {
    int32_t tc_fwd_ctas;       /* tensor-core forward with tc_fwd_split = 0: persistent CTAs per SM, 1, 2 or 3 */
    int32_t tc_fwd_levels;     /* tensor-core forward: levels whose corner loads a gathering thread issues
                                  together, 1 or 2 */
    int32_t fp32_ctas;         /* binary32 field kernels: persistent CTAs per SM, 1 or 2 */
    int32_t composite_threads; /* compositing kernel: threads per block, 64..512, multiple of 32 */
    int32_t sampler_threads;   /* ray and sample kernels: threads per block, 128..512, multiple of 32 */
    int32_t tuned;             /* out: 1 if the values came from snk_autotune */
    int32_t tc_bwd_saved;      /* tensor-core training step: 1 (default) the forward stores each layer's
                                  activations (FP16 high parts, 544 B a sample with a colour network, 576 B
                                  with view directions, 256 B without) in a context-owned buffer sized for
                                  the reserved samples, and the backward copies them back instead of
                                  recomputing the forward, when that buffer fits the context's
                                  activation budget (snk_ctx_set_act_budget) and can be allocated --
                                  else the step recomputes them; 0 the backward recomputes them.  Same
                                  results either way (up to the order of float atomics);
                                  snk_state.bwd_mode records which ran. */
    int32_t tc_fwd_split;      /* tensor-core forward: 1 (default) eight gather warps a CTA interpolate the
                                  next tile's features while four MMA / epilogue warps run the current
                                  tile's MLP chain, two CTAs per SM (tc_fwd_ctas unused); 0 every thread
                                  gathers a tile's features, then runs its chain (tc_fwd_ctas CTAs per
                                  SM).  Either with tc_fwd_levels; both unused by the E4M3 model. */
} snk_tuning;

/* Current launch shapes of ctx (defaults until tuned or set). */
int snk_get_tuning(snk_ctx *ctx, snk_tuning *out);
/* Set the launch shapes of ctx (tuned is ignored); SNK_ERR_INVALID_ARG for a value out of range. */
int snk_set_tuning(snk_ctx *ctx, const snk_tuning *in);
/* Autotuner: time every candidate launch shape of the sampler, field-forward,
 * field-backward (binary32 path) and compositing kernels on this batch (CUDA
 * events on `stream`, one warm-up run and one or two timed runs each, one
 * stage at a time; tensor cores: per backward mode the fastest forward of
 * tc_fwd_split 1, and 0 at 1, 2 or 3 CTAs per SM, each at 1 or 2 levels,
 * then forward + backward pick the mode) and keep the fastest for every
 * later call on ctx.  Reads
 * p->params / p->params_lp only: the caller's gradients, Adam state and step
 * state are untouched (the tuner allocates its own scratch gradient buffer and
 * state, and frees them).  Synchronises the stream; not graph-capturable.
 * out (nullable) receives the chosen shapes. */
int snk_autotune(snk_ctx *ctx, const snk_model *model, const snk_window *win, const uint32_t *pix, int B,
                 const snk_sampler *sampler, const snk_params *p, snk_stream_t stream, snk_tuning *out);

/* ---- diagnostics -------------------------------------------------------- */

/* Host only: number of kernels libsnk has launched in this process. */
int64_t snk_launch_count(void);
/* enable != 0: snk_train_step and snk_render record CUDA events on their
 * stream around each stage (0 rays/segments/samples, 1 field forward,
 * 2 rendering + loss + rendering backward, 3 field backward, 4 Adam).
 * Enabling (again) clears what was recorded. */
int snk_stage_timing(snk_ctx *ctx, int enable);
/* Synchronise and return, per stage, the summed milliseconds and the number
 * of recorded calls since timing was enabled (ms, calls: n entries, n <= 5). */
int snk_stage_times(snk_ctx *ctx, double *ms, int64_t *calls, int n);

/* Reduction-rate probe (the paper has no counterpart: it measures the peak of the
 * roofline that binds the hash-table gradient scatter).  Adds 1.0f with n_ops
 * fire-and-forget reductions to slots of table, a caller-owned device array of
 * n16 16-byte slots (n16 x 4 binary32, 16-byte aligned): operation i targets
 * slot floor(h(i) n16 / 2^32), h a 32-bit multiplicative hash of i + seed, as
 * one red.global.add.v4.f32 on the whole slot (width 16) or one .v2.f32 on half
 * i mod 2 of it (width 8).  Nothing else runs in the kernel (full occupancy,
 * grid-stride loop), so the caller's CUDA-event time of the call is the GPU's
 * reduction rate for random addresses in a table of that size.  The table's sum
 * grows by n_ops x width / 4.  SNK_ERR_INVALID_ARG for a NULL or misaligned
 * table, n16 outside 1..2^32-1, n_ops < 0 or another width.  Asynchronous. */
int snk_l2_reduction_probe(snk_ctx *ctx, float *table, int64_t n16, int64_t n_ops, int width, uint32_t seed,
                           snk_stream_t stream);

/* Wait for `stream` and report device-side status bits of `state` as a
 * status code (SNK_ERR_DEVICE_CHECK, SNK_ERR_TIMEOUT, SNK_ERR_OVERFLOW). */
int snk_sync_status(snk_ctx *ctx, const snk_state *state, snk_stream_t stream);

/* Self-test of the bounded device waits (every mbarrier wait of the tensor-core
 * field kernels gives up after 2 s, sets the timeout bit of the step state and
 * returns): one CTA waits on an mbarrier that receives its arrival (arrive != 0:
 * the wait completes, state unchanged) or never does (arrive == 0: after 2 s the
 * timeout bit is set, so snk_sync_status returns SNK_ERR_TIMEOUT, and the context
 * stays usable).  state: device snk_state (not cleared here).  Asynchronous. */
int snk_wait_selftest(snk_ctx *ctx, int arrive, snk_state *state, snk_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* SNK_H */
