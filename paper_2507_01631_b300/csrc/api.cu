// C ABI of libsnk: context and workspace, argument validation, host-side
// model layout, and the order of the kernels of one training step.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <algorithm>
#include <atomic>
#include <vector>

#include "kernels.cuh"

namespace snk {
std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace snk

struct snk_ctx {
  int device = 0;
  int sm_count = 148;
  char err[512] = {0};
  int64_t cap_rays = 0, cap_samples = 0;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  snk::RayBuffers rb{};
  float *sigma_rgb = nullptr;  // [cap_samples][4]
  float *dsr = nullptr;        // [cap_samples][4]
  uint16_t *feat_lp = nullptr; // [cap_samples + 128][2][32] FP16 features (high, low parts), mixed path;
                               // the E4M3 path uses the same bytes as [cap_samples + 128][32] binary32 features
  uint8_t *codes = nullptr;    // [cap_samples + 128][32] E4M3 first-layer codes
  uint32_t *amax = nullptr;    // [4] per-slot max |feature| (binary32 bits), E4M3 path
  snk::Tuning tune;            // launch shapes (snk_autotune / snk_set_tuning)
  bool tuned = false;
  void *pool_ws = nullptr;     // ray pool scratch: base [kMaxViews + 1] i64 | chunk counts | pixel flags
  size_t pool_ws_bytes = 0;
  void *occ_ws = nullptr;      // occupancy update scratch: state | per-block partial sums | thresholds
  size_t occ_ws_bytes = 0;
  void *acts = nullptr;        // stored activations of a tensor-core training step (tc_bwd_saved)
  size_t acts_bytes = 0;
  int64_t act_budget = -1;     // most bytes acts may take (snk_ctx_set_act_budget); < 0: no budget
  uint16_t *cells_lp = nullptr;  // mixed path: cell-major FP16 copy of the dense levels (rewritten before a forward)
  size_t cells_lp_bytes = 0;
  float *cell_grad = nullptr;    // mixed path: cell-major gradients of the dense levels (zero between steps)
  size_t cell_grad_bytes = 0;
  snk::DevView *d_views = nullptr;
  snk::DevView *h_views = nullptr;  // pinned staging
  int n_views = 0;
  // stage timing (diagnostics)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> recorded;
  size_t ev_used = 0;
};

namespace {
cudaEvent_t next_event(snk_ctx *c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

// Records the start of a stage; stage_end() records its end.
struct StageMark {
  snk_ctx *c;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageMark(snk_ctx *c_, int s, cudaStream_t st_) : c(c_), stage(s), st(st_) {
    if (c->timing && (a = next_event(c))) cudaEventRecord(a, st);
  }
  ~StageMark() {
    if (!a) return;
    cudaEvent_t b = next_event(c);
    if (!b) return;
    cudaEventRecord(b, st);
    c->recorded.push_back({stage, {a, b}});
  }
};
}  // namespace

namespace {

using namespace snk;

int fail(snk_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define SNK_CK(ctx, call)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(ctx, SNK_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int layout_of(const snk_model *m, snk_layout *o, char *msg, size_t msg_len) {
  auto bad = [&](const char *why) {
    snprintf(msg, msg_len, "invalid model: %s", why);
    return SNK_ERR_INVALID_ARG;
  };
  if (!m || !o) return bad("NULL pointer");
  if (m->L < 1 || m->L > kMaxLevels) return bad("L must be in 1..32");
  if (m->F != 2) return bad("F must be 2");
  const int in = m->L * m->F;
  if (in != 8 && in != 16 && in != 32) return bad("L*F must be 8, 16 or 32");
  if (m->log2_T < 4 || m->log2_T > 24) return bad("log2_T must be in 4..24");
  if (m->n_min < 2 || m->n_max < m->n_min || m->n_max > 4095) return bad("need 2 <= n_min <= n_max < 4096");
  if (m->hidden != kHidden) return bad("hidden must be 64");
  if (m->colour != 0 && m->colour != 1) return bad("colour must be 0 or 1");
  if (m->geo_out != (m->colour ? 16 : 4)) return bad("geo_out must be 16 with a colour MLP, 4 without");
  if (m->shared_colour != 0 && m->shared_colour != 1) return bad("shared_colour must be 0 or 1");
  if (m->n_slots < 1 || m->n_slots > kMaxSlots) return bad("n_slots must be in 1..4");
  if (m->precision != SNK_FP32 && m->precision != SNK_MIXED && m->precision != SNK_MIXED_E4M3)
    return bad("precision must be SNK_FP32, SNK_MIXED or SNK_MIXED_E4M3");
  if (m->view_dirs != 0 && m->view_dirs != 1) return bad("view_dirs must be 0 or 1");
  if (m->view_dirs && !m->colour) return bad("view_dirs needs a colour MLP");
  if (m->view_dirs && m->precision == SNK_MIXED_E4M3) return bad("view_dirs is not available with SNK_MIXED_E4M3");
  memset(o, 0, sizeof(*o));
  const int64_t T = (int64_t)1 << m->log2_T;
  const double b = m->L > 1 ? std::exp((std::log((double)m->n_max) - std::log((double)m->n_min)) / (m->L - 1)) : 1.0;
  int64_t off = 0;
  for (int l = 0; l < m->L; ++l) {
    const int64_t res = (int64_t)std::floor((double)m->n_min * std::pow(b, (double)l) + 1e-6);
    const int64_t nv = (res + 1) * (res + 1) * (res + 1);
    const bool dense = nv <= T;
    int64_t size = dense ? nv : T;
    size = (size + 7) / 8 * 8;
    o->res[l] = (int32_t)res;
    o->dense[l] = dense ? 1 : 0;
    o->level_offset[l] = off;
    o->level_size[l] = size;
    off += size;
  }
  o->n_entries = off;
  o->grid_params = off * m->F;
  const int64_t geo = (int64_t)kHidden * in + (int64_t)kHidden * kHidden + (int64_t)m->geo_out * kHidden;
  o->tile_params = o->grid_params + geo;
  const int64_t col_in = m->geo_out + (m->view_dirs ? 16 : 0);
  o->colour_params = m->colour ? (int64_t)kHidden * col_in + (int64_t)kHidden * kHidden + 3 * kHidden : 0;
  o->n_colour_blocks = m->colour ? (m->shared_colour ? 1 : m->n_slots) : 0;
  o->n_params = m->n_slots * o->tile_params + o->n_colour_blocks * o->colour_params;
  o->n_optimisers = m->n_slots + o->n_colour_blocks;
  return SNK_OK;
}

ModelDev model_dev(const snk_model *m, const snk_layout &lay) {
  ModelDev d{};
  d.grid.L = m->L;
  d.grid.F = m->F;
  d.grid.log2_T = m->log2_T;
  d.grid.T = 1 << m->log2_T;
  uint32_t cells = 0;
  for (int l = 0; l < m->L; ++l) {
    d.grid.res[l] = lay.res[l];
    d.grid.dense[l] = lay.dense[l];
    d.grid.offset[l] = (uint32_t)lay.level_offset[l];
    d.grid.cell_off[l] = cells;
    if (lay.dense[l]) {
      cells += (uint32_t)lay.res[l] * (uint32_t)lay.res[l] * (uint32_t)lay.res[l];
      d.grid.dense_end = (uint32_t)(lay.level_offset[l] + lay.level_size[l]);
    }
  }
  d.grid.n_cells = cells;
  d.in_dim = m->L * m->F;
  d.geo_out = m->geo_out;
  d.colour = m->colour;
  d.shared_colour = m->shared_colour;
  d.n_slots = m->n_slots;
  d.mixed = m->precision != SNK_FP32;
  d.e4m3 = m->precision == SNK_MIXED_E4M3;
  d.view_dirs = m->view_dirs;
  d.col_in = m->geo_out + (m->view_dirs ? 16 : 0);
  d.tile_params = lay.tile_params;
  d.grid_params = lay.grid_params;
  d.colour_params = lay.colour_params;
  d.colour_base = (int64_t)m->n_slots * lay.tile_params;
  d.w1 = lay.grid_params;
  d.w2 = d.w1 + (int64_t)kHidden * d.in_dim;
  d.w3 = d.w2 + (int64_t)kHidden * kHidden;
  d.v1 = 0;
  d.v2 = (int64_t)kHidden * d.col_in;
  d.v3 = d.v2 + (int64_t)kHidden * kHidden;
  return d;
}

// The context's error text as the message sink of the shared descriptor checks.
ErrSink sink(snk_ctx *ctx) { return ErrSink{ctx ? ctx->err : nullptr, ctx ? sizeof(ctx->err) : 0}; }

size_t carve(size_t &off, size_t bytes) {
  const size_t o = off;
  off += (bytes + 255) / 256 * 256;
  return o;
}

// Lay the workspace out for B rays and S samples; with base == nullptr only sizes it.
size_t layout_ws(snk_ctx *ctx, char *base, int64_t B, int64_t S) {
  size_t off = 0;
  const int64_t nb = scan_blocks((int)B > 0 ? (int)B : 1);
  RayBuffers rb{};
  rb.ray_od = (float *)(base + carve(off, sizeof(float) * 6 * B));
  rb.ray_ok = (uint8_t *)(base + carve(off, B));
  rb.seg_slot = (uint8_t *)(base + carve(off, 3 * B));
  rb.seg_t = (float *)(base + carve(off, sizeof(float) * 6 * B));
  rb.seg_n = (uint32_t *)(base + carve(off, sizeof(uint32_t) * 3 * B));
  rb.seg_off = (uint32_t *)(base + carve(off, sizeof(uint32_t) * 3 * B));
  rb.seg_k = (uint32_t *)(base + carve(off, sizeof(uint32_t) * 3 * B));
  rb.cnt = (uint32_t *)(base + carve(off, sizeof(uint32_t) * 5 * B));
  rb.excl = (uint32_t *)(base + carve(off, sizeof(uint32_t) * 5 * B));
  rb.block_tot = (uint32_t *)(base + carve(off, sizeof(uint32_t) * 5 * nb));
  rb.smp_t = (float *)(base + carve(off, sizeof(float) * S));
  rb.smp_dt = (float *)(base + carve(off, sizeof(float) * S));
  rb.smp_xyz = (float *)(base + carve(off, sizeof(float) * 3 * S));
  rb.smp_ray = (uint32_t *)(base + carve(off, sizeof(uint32_t) * S));
  float *sr = (float *)(base + carve(off, sizeof(float) * 4 * S));
  float *dsr = (float *)(base + carve(off, sizeof(float) * 4 * S));
  uint16_t *flp = (uint16_t *)(base + carve(off, sizeof(uint16_t) * 64 * (S + 128)));
  uint8_t *codes = (uint8_t *)(base + carve(off, (size_t)32 * (S + 128)));
  uint32_t *amax = (uint32_t *)(base + carve(off, sizeof(uint32_t) * kMaxSlots));
  if (base) {
    ctx->rb = rb;
    ctx->sigma_rgb = sr;
    ctx->dsr = dsr;
    ctx->feat_lp = flp;
    ctx->codes = codes;
    ctx->amax = amax;
  }
  return off;
}

int ensure_ws(snk_ctx *ctx, int64_t B, int64_t S) {
  if (B <= ctx->cap_rays && S <= ctx->cap_samples && ctx->ws) return SNK_OK;
  const int64_t nB = B > ctx->cap_rays ? B : ctx->cap_rays;
  const int64_t nS = S > ctx->cap_samples ? S : ctx->cap_samples;
  const size_t bytes = layout_ws(ctx, nullptr, nB, nS);
  if (ctx->ws) {
    SNK_CK(ctx, cudaDeviceSynchronize());
    SNK_CK(ctx, cudaFree(ctx->ws));
    ctx->ws = nullptr;
  }
  if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    ctx->cap_rays = ctx->cap_samples = 0;
    return fail(ctx, SNK_ERR_OOM, "workspace of %zu bytes (%lld rays, %lld samples) could not be allocated", bytes,
                (long long)nB, (long long)nS);
  }
  ctx->ws_bytes = bytes;
  ctx->cap_rays = nB;
  ctx->cap_samples = nS;
  layout_ws(ctx, (char *)ctx->ws, nB, nS);
  return SNK_OK;
}

// Samples of a batch of B rays at most.  Uniform mode: K_ray a ray.  Otherwise a ray's segments
// take K = clamp(rint(K_ray len_seg / len_ray), K_min, K_max) each: the segments above K_min share
// at most K_ray (plus 1/2 of rounding each and a few binary32 ulps of the shares' sum), so a ray
// holds at most max(segs K_min, (segs - 1) K_min + K_ray) + segs samples, and segs K_max.  A batch
// that still overflowed would set the status check bit and produce no samples.
int64_t max_samples_for(const snk_window *w, const snk_sampler *s, int64_t B) {
  const int64_t segs = 1 + (w->nx == 2 ? 1 : 0) + (w->ny == 2 ? 1 : 0);
  int64_t per_ray = s->K_ray;
  if (s->mode != kSampleUniform) {
    const int64_t shares = std::max<int64_t>(segs * s->K_min, (segs - 1) * s->K_min + s->K_ray) + segs;
    per_ray = std::min<int64_t>(segs * s->K_max, shares);
  }
  return B * per_ray + (int64_t)kSlotAlign * kMaxSlots;
}

// Bytes of the stored-activation buffer of a tensor-core training step for the context's
// sample capacity.
size_t acts_need(const snk_ctx *ctx, const snk_model *model) {
  return (size_t)(ctx->cap_samples / 128 + 1) * (size_t)act_tile_bytes(model->colour != 0, model->view_dirs != 0);
}

// The stored-activation buffer for the context's capacity, or nullptr when it exceeds the
// activation budget or cannot be allocated: the step then recomputes the activations in its
// backward (the per-sample activations are recomputed instead of stored when the batch
// outgrows memory).  Not an error: nothing is written to the context's error text.
uint16_t *acts_or_recompute(snk_ctx *ctx, const snk_model *model, cudaStream_t st) {
  const size_t need = acts_need(ctx, model);
  if (ctx->act_budget >= 0 && need > (size_t)ctx->act_budget) return nullptr;
  if (need <= ctx->acts_bytes) return static_cast<uint16_t *>(ctx->acts);
  if (ctx->acts) {
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cudaFree(ctx->acts);
    ctx->acts = nullptr;
    ctx->acts_bytes = 0;
  }
  if (cudaMalloc(&ctx->acts, need) != cudaSuccess) {
    cudaGetLastError();  // not sticky: the recompute backward runs instead
    ctx->acts = nullptr;
    return nullptr;
  }
  ctx->acts_bytes = need;
  return static_cast<uint16_t *>(ctx->acts);
}

// The cell-major buffers of the dense levels for a mixed model (cells.cu): the FP16 copy the
// forward gathers from and the gradient accumulator the backward scatters into.  A buffer that
// cannot be allocated is not an error: the field kernels then use the table (and its gradient)
// directly, with the same results.  The accumulator is cleared when allocated and kept clear by the
// fold after each backward.
uint16_t *cells_lp_for(snk_ctx *ctx, const ModelDev &md) {
  const size_t need = (size_t)md.n_slots * md.grid.n_cells * 32;
  if (need == 0) return nullptr;
  if (need <= ctx->cells_lp_bytes) return ctx->cells_lp;
  if (ctx->cells_lp) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cudaFree(ctx->cells_lp);
    ctx->cells_lp = nullptr;
    ctx->cells_lp_bytes = 0;
  }
  if (cudaMalloc(&ctx->cells_lp, need) != cudaSuccess) {
    cudaGetLastError();
    ctx->cells_lp = nullptr;
    return nullptr;
  }
  ctx->cells_lp_bytes = need;
  return ctx->cells_lp;
}

float *cell_grad_for(snk_ctx *ctx, const ModelDev &md, cudaStream_t st) {
  const size_t need = (size_t)md.n_slots * md.grid.n_cells * 64;
  if (need == 0) return nullptr;
  if (need <= ctx->cell_grad_bytes) return ctx->cell_grad;
  if (ctx->cell_grad) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cudaFree(ctx->cell_grad);
    ctx->cell_grad = nullptr;
    ctx->cell_grad_bytes = 0;
  }
  if (cudaMalloc(&ctx->cell_grad, need) != cudaSuccess) {
    cudaGetLastError();
    ctx->cell_grad = nullptr;
    return nullptr;
  }
  if (cudaMemsetAsync(ctx->cell_grad, 0, need, st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->cell_grad);
    ctx->cell_grad = nullptr;
    return nullptr;
  }
  ctx->cell_grad_bytes = need;
  return ctx->cell_grad;
}

int prepare(snk_ctx *ctx, const snk_model *model, snk_layout *lay, ModelDev *md) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  const int rc = layout_of(model, lay, ctx->err, sizeof(ctx->err));
  if (rc != SNK_OK) return rc;
  *md = model_dev(model, *lay);
  return SNK_OK;
}

int check_params(snk_ctx *ctx, const snk_model *model, const snk_params *p, bool train) {
  if (!p || !p->params) return fail(ctx, SNK_ERR_INVALID_ARG, "params is NULL");
  if (model->precision != SNK_FP32 && !p->params_lp)
    return fail(ctx, SNK_ERR_INVALID_ARG, "mixed precision needs the params_lp working copy");
  if (train && (!p->grads || !p->adam_m || !p->adam_v || !p->adam_step))
    return fail(ctx, SNK_ERR_INVALID_ARG, "training needs grads, adam_m, adam_v and adam_step");
  return SNK_OK;
}

}  // namespace

extern "C" {

const char *snk_version(void) { return "libsnk 0.1 (sm_103a)"; }

int64_t snk_max_samples(const snk_window *win, const snk_sampler *sampler, int64_t B) {
  if (!win || !sampler || B < 0) return -1;
  return max_samples_for(win, sampler, B);
}

int snk_abi_sizes(int64_t *sizes, int n) {
  const int64_t all[9] = {(int64_t)sizeof(snk_camera), (int64_t)sizeof(snk_window), (int64_t)sizeof(snk_model),
                          (int64_t)sizeof(snk_layout), (int64_t)sizeof(snk_sampler), (int64_t)sizeof(snk_adam),
                          (int64_t)sizeof(snk_params), (int64_t)sizeof(snk_state), (int64_t)sizeof(snk_tuning)};
  if (!sizes || n < 0) return 0;
  const int k = n < 9 ? n : 9;
  for (int i = 0; i < k; ++i) sizes[i] = all[i];
  return k;
}

int snk_model_layout(const snk_model *model, snk_layout *out) {
  char msg[256];
  return layout_of(model, out, msg, sizeof(msg));
}

int snk_ctx_create(int device, snk_ctx **out) {
  if (!out) return SNK_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return SNK_ERR_CUDA;
  }
  snk_ctx *c = new snk_ctx();
  c->device = device;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
    c->sm_count = sms;
  if (cudaMalloc(&c->d_views, sizeof(DevView) * kMaxViews) != cudaSuccess ||
      cudaMallocHost(&c->h_views, sizeof(DevView) * kMaxViews) != cudaSuccess) {
    cudaGetLastError();
    if (c->d_views) cudaFree(c->d_views);
    delete c;
    return SNK_ERR_OOM;
  }
  *out = c;
  return SNK_OK;
}

int snk_ctx_destroy(snk_ctx *ctx) {
  if (!ctx) return SNK_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->pool_ws) cudaFree(ctx->pool_ws);
  if (ctx->occ_ws) cudaFree(ctx->occ_ws);
  if (ctx->acts) cudaFree(ctx->acts);
  if (ctx->cells_lp) cudaFree(ctx->cells_lp);
  if (ctx->cell_grad) cudaFree(ctx->cell_grad);
  if (ctx->d_views) cudaFree(ctx->d_views);
  if (ctx->h_views) cudaFreeHost(ctx->h_views);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
  return SNK_OK;
}

int snk_ctx_reserve(snk_ctx *ctx, int64_t max_rays, int64_t max_samples) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (max_rays < 1 || max_rays > (1 << 22) || max_samples < 0 || max_samples > 0xFFFFFF00ll)
    return fail(ctx, SNK_ERR_INVALID_ARG, "reserve: need 1 <= max_rays <= 2^22 and 0 <= max_samples < 2^32");
  return ensure_ws(ctx, max_rays, max_samples);
}

int snk_ctx_set_act_budget(snk_ctx *ctx, int64_t bytes) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  ctx->act_budget = bytes < 0 ? -1 : bytes;
  if (ctx->acts && bytes >= 0 && ctx->acts_bytes > (size_t)bytes) {
    SNK_CK(ctx, cudaDeviceSynchronize());
    SNK_CK(ctx, cudaFree(ctx->acts));
    ctx->acts = nullptr;
    ctx->acts_bytes = 0;
  }
  return SNK_OK;
}

const char *snk_last_error(const snk_ctx *ctx) { return ctx ? ctx->err : "NULL context"; }

int snk_params_refresh_lp(snk_ctx *ctx, const snk_model *model, const snk_params *p, snk_stream_t stream) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  if (model->precision == SNK_FP32) return fail(ctx, SNK_ERR_INVALID_ARG, "snk_params_refresh_lp: a binary32 model has no working copy");
  if (!p || !p->params || !p->params_lp) return fail(ctx, SNK_ERR_INVALID_ARG, "snk_params_refresh_lp: NULL params or params_lp");
  SNK_CK(ctx, launch_refresh_lp(p->params, p->params_lp, lay.n_params, ctx->sm_count, (cudaStream_t)stream));
  return SNK_OK;
}

int snk_set_views(snk_ctx *ctx, const snk_camera *cams, int n_views, const float *const *crops, snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (!cams || n_views < 1 || n_views > kMaxViews)
    return fail(ctx, SNK_ERR_INVALID_ARG, "need 1..%d cameras", kMaxViews);
  SNK_CK(ctx, cudaStreamSynchronize((cudaStream_t)stream));  // the staging buffer may still be in flight
  for (int v = 0; v < n_views; ++v) {
    const int rc = check_camera(sink(ctx), cams[v], v, &ctx->h_views[v]);
    if (rc != SNK_OK) return rc;
    ctx->h_views[v].crop = crops ? crops[v] : nullptr;
  }
  SNK_CK(ctx, cudaMemcpyAsync(ctx->d_views, ctx->h_views, sizeof(DevView) * n_views, cudaMemcpyHostToDevice,
                              (cudaStream_t)stream));
  SNK_CK(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  ctx->n_views = n_views;
  return SNK_OK;
}

int snk_sample_segments(snk_ctx *ctx, const snk_window *win, const uint32_t *pix, int B, const snk_sampler *sampler,
                        float *ray_od, uint8_t *ray_ok, uint8_t *seg_slot, float *seg_t, uint32_t *seg_n,
                        uint32_t *seg_off, float *smp_t, float *smp_dt, float *smp_xyz, int64_t cap, snk_state *state,
                        snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (B < 0 || B > (1 << 22)) return fail(ctx, SNK_ERR_INVALID_ARG, "B must be in 0..2^22");
  if (!win) return fail(ctx, SNK_ERR_INVALID_ARG, "window is NULL");
  WinParams wp;
  int rc = check_window(sink(ctx), win, win->nx * win->ny, &wp);
  if (rc) return rc;
  SamplerParams sp;
  if ((rc = check_sampler(sink(ctx), sampler, &sp))) return rc;
  if (ctx->n_views < 1) return fail(ctx, SNK_ERR_INVALID_ARG, "no views: call snk_set_views first");
  if (B > 0 && (!pix || !ray_od || !ray_ok || !seg_slot || !seg_t || !seg_n || !seg_off || !smp_t || !smp_dt ||
                !smp_xyz || !state))
    return fail(ctx, SNK_ERR_INVALID_ARG, "NULL buffer");
  if ((rc = ensure_ws(ctx, B > 0 ? B : 1, ctx->cap_samples))) return rc;
  RayBuffers rb = ctx->rb;
  rb.ray_od = ray_od;
  rb.ray_ok = ray_ok;
  rb.seg_slot = seg_slot;
  rb.seg_t = seg_t;
  rb.seg_n = seg_n;
  rb.seg_off = seg_off;
  rb.smp_t = smp_t;
  rb.smp_dt = smp_dt;
  rb.smp_xyz = smp_xyz;
  rb.smp_ray = nullptr;  // caller-sized buffers: the workspace's per-sample ray index may be shorter than cap
  SNK_CK(ctx, launch_sample_segments(ctx->d_views, ctx->n_views, wp, sp, pix, B, 0, rb, cap, state,
                                     (cudaStream_t)stream, ctx->tune));
  return SNK_OK;
}

int snk_encode(snk_ctx *ctx, const snk_model *model, const snk_params *p, const float *smp_xyz,
               const snk_state *state, int64_t S, float *feat, uint32_t *idx_out, snk_stream_t stream) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  if (!p || !p->params || !smp_xyz || !state || !feat || S < 0)
    return fail(ctx, SNK_ERR_INVALID_ARG, "NULL buffer or negative S");
  FieldArgs fa{};
  fa.m = md;
  fa.params = p->params;
  fa.xyz = smp_xyz;
  fa.feat_out = feat;
  fa.idx_out = idx_out;
  fa.state = state;
  fa.S = S;
  fa.slot_only = -1;
  fa.mode = kEncodeOnly;
  SNK_CK(ctx, launch_field_fp32(fa, ctx->sm_count, (cudaStream_t)stream, ctx->tune));
  return SNK_OK;
}

int snk_encode_backward(snk_ctx *ctx, const snk_model *model, const snk_params *p, const float *smp_xyz,
                        const snk_state *state, int64_t S, const float *dfeat, snk_stream_t stream) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  if (!p || !p->grads || !smp_xyz || !state || !dfeat || S < 0)
    return fail(ctx, SNK_ERR_INVALID_ARG, "NULL buffer or negative S");
  FieldArgs fa{};
  fa.m = md;
  fa.grads = p->grads;
  fa.xyz = smp_xyz;
  fa.feat_in = dfeat;
  fa.state = state;
  fa.S = S;
  fa.slot_only = -1;
  SNK_CK(ctx, launch_encode_scatter(fa, (cudaStream_t)stream));
  return SNK_OK;
}

int snk_mlp(snk_ctx *ctx, const snk_model *model, const snk_params *p, const float *feat, const snk_state *state,
            int64_t S, float *out, snk_stream_t stream) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  if (!p || !p->params || !feat || !state || !out || S < 0)
    return fail(ctx, SNK_ERR_INVALID_ARG, "NULL buffer or negative S");
  if (model->view_dirs)
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_mlp: the view-direction colour input needs the rays; use the step entry points");
  FieldArgs fa{};
  fa.m = md;
  fa.params = p->params;
  fa.feat_in = feat;
  fa.sigma_rgb = out;
  fa.state = state;
  fa.S = S;
  fa.slot_only = -1;
  fa.mode = kForward;
  SNK_CK(ctx, launch_field_fp32(fa, ctx->sm_count, (cudaStream_t)stream, ctx->tune));
  return SNK_OK;
}

int snk_mlp_backward(snk_ctx *ctx, const snk_model *model, const snk_params *p, const float *feat,
                     const snk_state *state, int64_t S, const float *dout, float *dfeat, snk_stream_t stream) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  if (!p || !p->params || !p->grads || !feat || !state || !dout || !dfeat || S < 0)
    return fail(ctx, SNK_ERR_INVALID_ARG, "NULL buffer or negative S");
  if (model->view_dirs)
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_mlp_backward: the view-direction colour input needs the rays; use the step entry points");
  FieldArgs fa{};
  fa.m = md;
  fa.params = p->params;
  fa.grads = p->grads;
  fa.feat_in = feat;
  fa.dsr = dout;
  fa.dfeat_out = dfeat;
  fa.state = state;
  fa.S = S;
  fa.slot_only = -1;
  fa.mode = kBackward;
  SNK_CK(ctx, launch_field_fp32(fa, ctx->sm_count, (cudaStream_t)stream, ctx->tune));
  return SNK_OK;
}

int snk_composite(snk_ctx *ctx, const float *sigma_rgb, const float *smp_t, const float *smp_dt,
                  const uint32_t *seg_n, const uint32_t *seg_off, int B, float *out, float *t_final,
                  snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (B < 0 || (B > 0 && (!sigma_rgb || !smp_t || !smp_dt || !seg_n || !seg_off || !out)))
    return fail(ctx, SNK_ERR_INVALID_ARG, "NULL buffer or negative B");
  CompositeArgs ca{};
  ca.sigma_rgb = sigma_rgb;
  ca.smp_t = smp_t;
  ca.smp_dt = smp_dt;
  ca.seg_n = seg_n;
  ca.seg_off = seg_off;
  ca.B = B;
  ca.out = out;
  ca.t_final = t_final;
  SNK_CK(ctx, launch_composite(ca, (cudaStream_t)stream, ctx->tune));
  return SNK_OK;
}

int snk_composite_backward(snk_ctx *ctx, const float *sigma_rgb, const float *smp_t, const float *smp_dt,
                           const uint32_t *seg_n, const uint32_t *seg_off, int B, const float *g_rgb,
                           float *d_sigma_rgb, snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (B < 0 || (B > 0 && (!sigma_rgb || !smp_t || !smp_dt || !seg_n || !seg_off || !g_rgb || !d_sigma_rgb)))
    return fail(ctx, SNK_ERR_INVALID_ARG, "NULL buffer or negative B");
  CompositeArgs ca{};
  ca.sigma_rgb = sigma_rgb;
  ca.smp_t = smp_t;
  ca.smp_dt = smp_dt;
  ca.seg_n = seg_n;
  ca.seg_off = seg_off;
  ca.B = B;
  ca.g_rgb = g_rgb;
  ca.dsr = d_sigma_rgb;
  SNK_CK(ctx, launch_composite(ca, (cudaStream_t)stream, ctx->tune));
  return SNK_OK;
}

// The workspace's ray buffers for a step of `model`: the per-sample ray index is written only
// when the colour input needs the view direction.
static RayBuffers step_rays(const snk_ctx *ctx, const snk_model *model) {
  RayBuffers rb = ctx->rb;
  if (!model->view_dirs) rb.smp_ray = nullptr;
  return rb;
}

// n_rays: the batch size of the rays whose directions ray_od holds ([6][n_rays]); every
// sample's ray index (rb.smp_ray) is below it.
// acts: a training step's stored-activation buffer (its forward writes it, its backward reads
// it back), or nullptr: no stored activations (the backward recomputes them).  Decided once
// per step, so that the forward and backward of a step agree.
static int run_field(snk_ctx *ctx, const snk_model *model, const ModelDev &md, const snk_params *p,
                     const snk_state *state, int mode, cudaStream_t st, int n_rays, uint16_t *acts) {
  FieldArgs fa{};
  fa.m = md;
  fa.params = p->params;
  fa.params_lp = p->params_lp;
  fa.grads = p->grads;
  fa.xyz = ctx->rb.smp_xyz;
  fa.sigma_rgb = ctx->sigma_rgb;
  fa.dsr = ctx->dsr;
  fa.feat_lp = ctx->feat_lp;
  fa.feat32 = reinterpret_cast<float *>(ctx->feat_lp);
  fa.codes = ctx->codes;
  fa.amax = ctx->amax;
  fa.state = state;
  fa.S = ctx->cap_samples;
  fa.mode = mode;
  fa.smp_ray = ctx->rb.smp_ray;
  fa.ray_od = ctx->rb.ray_od;
  fa.n_rays = n_rays;
  if (model->precision != SNK_FP32) {
    fa.slot_only = -1;
    fa.acts = acts;
    if (md.e4m3 && mode == kForward) {
      // the per-slot scales need every feature of the batch first
      SNK_CK(ctx, cudaMemsetAsync(ctx->amax, 0, sizeof(uint32_t) * kMaxSlots, st));
      SNK_CK(ctx, launch_gather_amax(fa, ctx->sm_count, st));
    }
    if (mode == kForward && !md.e4m3 && (fa.cells_lp = cells_lp_for(ctx, md)) != nullptr)
      SNK_CK(ctx, launch_cells_copy(p->params_lp, md.tile_params, md.grid, md.n_slots, ctx->cells_lp, ctx->sm_count, st));
    if (mode == kBackward) fa.cell_grad = cell_grad_for(ctx, md, st);
    SNK_CK(ctx, launch_field_tc(fa, ctx->sm_count, st, ctx->tune));
    if (fa.cell_grad)
      SNK_CK(ctx, launch_cells_fold(fa.cell_grad, p->grads, md.tile_params, md.grid, md.n_slots, ctx->sm_count, st));
    return SNK_OK;
  }
  // binary32 path: one launch chain per tile (slot), as a per-tile trainer issues them
  for (int k = 0; k < model->n_slots; ++k) {
    fa.slot_only = k;
    SNK_CK(ctx, launch_field_fp32(fa, ctx->sm_count, st, ctx->tune));
  }
  return SNK_OK;
}

int snk_train_step(snk_ctx *ctx, const snk_model *model, const snk_window *win, const uint32_t *pix, int B,
                   const snk_sampler *sampler, const snk_adam *adam, const snk_params *p, snk_state *state,
                   float *out, snk_stream_t stream) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  WinParams wp;
  if ((rc = check_window(sink(ctx), win, model->n_slots, &wp))) return rc;
  SamplerParams sp;
  if ((rc = check_sampler(sink(ctx), sampler, &sp))) return rc;
  sp.use_state_iteration = 1;
  sp.render = 0;
  if ((rc = check_params(ctx, model, p, true))) return rc;
  if (!adam) return fail(ctx, SNK_ERR_INVALID_ARG, "adam is NULL");
  if (!state || !pix || B < 1 || B > (1 << 22)) return fail(ctx, SNK_ERR_INVALID_ARG, "need state, pix, 1 <= B <= 2^22");
  if (ctx->n_views < 1) return fail(ctx, SNK_ERR_INVALID_ARG, "no views: call snk_set_views first");
  if ((rc = ensure_ws(ctx, B, max_samples_for(win, sampler, B)))) return rc;
  const cudaStream_t st = (cudaStream_t)stream;
  // backward mode of this step: stored activations when the buffer fits the budget and can be
  // had, else recomputed
  uint16_t *acts = nullptr;
  uint32_t bwd_mode = 0;
  if (model->precision != SNK_FP32) {
    if (ctx->tune.tc_bwd_saved) acts = acts_or_recompute(ctx, model, st);
    bwd_mode = acts ? 1u : 2u;
  }
  {
    StageMark m(ctx, 0, st);
    SNK_CK(ctx, launch_sample_segments(ctx->d_views, ctx->n_views, wp, sp, pix, B, 1, step_rays(ctx, model), ctx->cap_samples, state,
                                       st, ctx->tune));
  }
  {
    StageMark m(ctx, 1, st);
    if ((rc = run_field(ctx, model, md, p, state, kForward, st, B, acts))) return rc;
  }
  CompositeArgs ca{};
  ca.sigma_rgb = ctx->sigma_rgb;
  ca.smp_t = ctx->rb.smp_t;
  ca.smp_dt = ctx->rb.smp_dt;
  ca.seg_n = ctx->rb.seg_n;
  ca.seg_off = ctx->rb.seg_off;
  ca.B = B;
  ca.out = out;
  ca.pix = pix;
  ca.views = ctx->d_views;
  ca.dsr = ctx->dsr;
  ca.state = state;
  ca.train = 1;
  {
    StageMark m(ctx, 2, st);
    SNK_CK(ctx, launch_composite(ca, st, ctx->tune));
  }
  {
    StageMark m(ctx, 3, st);
    if ((rc = run_field(ctx, model, md, p, state, kBackward, st, B, acts))) return rc;
  }
  AdamArgs aa{};
  aa.params = p->params;
  aa.params_lp = p->params_lp;
  aa.grads = p->grads;
  aa.m = p->adam_m;
  aa.v = p->adam_v;
  aa.steps = p->adam_step;
  aa.n = lay.n_params;
  aa.n_groups = lay.n_optimisers;
  for (int k = 0; k < model->n_slots; ++k) {
    aa.start[k] = k * lay.tile_params;
    aa.end[k] = aa.start[k] + lay.tile_params;
    aa.mlp_start[k] = aa.start[k] + lay.grid_params;
  }
  for (int c = 0; c < lay.n_colour_blocks; ++c) {
    const int k = model->n_slots + c;
    aa.start[k] = md.colour_base + c * lay.colour_params;
    aa.end[k] = aa.start[k] + lay.colour_params;
    aa.mlp_start[k] = aa.start[k];
  }
  aa.lr = adam->lr;
  aa.beta1 = adam->beta1;
  aa.beta2 = adam->beta2;
  aa.eps = adam->eps;
  aa.l2 = adam->l2_mlp;
  aa.state = state;
  aa.mixed = model->precision != SNK_FP32;
  aa.bwd_mode = bwd_mode;
  {
    StageMark m(ctx, 4, st);
    SNK_CK(ctx, launch_adam(aa, ctx->sm_count, st));
  }
  return SNK_OK;
}

int snk_render(snk_ctx *ctx, const snk_model *model, const snk_window *win, const uint32_t *pix, int B,
               const snk_sampler *sampler, const snk_params *p, snk_state *state, float *out, snk_stream_t stream) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  WinParams wp;
  if ((rc = check_window(sink(ctx), win, model->n_slots, &wp))) return rc;
  SamplerParams sp;
  if ((rc = check_sampler(sink(ctx), sampler, &sp))) return rc;
  sp.render = 1;
  if ((rc = check_params(ctx, model, p, false))) return rc;
  if (!state || !pix || !out || B < 1 || B > (1 << 22))
    return fail(ctx, SNK_ERR_INVALID_ARG, "need state, pix, out and 1 <= B <= 2^22");
  if (ctx->n_views < 1) return fail(ctx, SNK_ERR_INVALID_ARG, "no views: call snk_set_views first");
  if ((rc = ensure_ws(ctx, B, max_samples_for(win, sampler, B)))) return rc;
  const cudaStream_t st = (cudaStream_t)stream;
  {
    StageMark m(ctx, 0, st);
    SNK_CK(ctx, launch_sample_segments(ctx->d_views, ctx->n_views, wp, sp, pix, B, 0, step_rays(ctx, model), ctx->cap_samples, state,
                                       st, ctx->tune));
  }
  {
    StageMark m(ctx, 1, st);
    if ((rc = run_field(ctx, model, md, p, state, kForward, st, B, nullptr))) return rc;
  }
  CompositeArgs ca{};
  ca.sigma_rgb = ctx->sigma_rgb;
  ca.smp_t = ctx->rb.smp_t;
  ca.smp_dt = ctx->rb.smp_dt;
  ca.seg_n = ctx->rb.seg_n;
  ca.seg_off = ctx->rb.seg_off;
  ca.B = B;
  ca.out = out;
  ca.state = state;
  {
    StageMark m(ctx, 2, st);
    SNK_CK(ctx, launch_composite(ca, st, ctx->tune));
  }
  return SNK_OK;
}

static bool tuning_ok(const snk_tuning &t) {
  auto mult32 = [](int v, int lo, int hi) { return v >= lo && v <= hi && v % 32 == 0; };
  return (t.tc_fwd_ctas >= 1 && t.tc_fwd_ctas <= 3) && (t.tc_fwd_levels == 1 || t.tc_fwd_levels == 2) &&
         (t.tc_bwd_saved == 0 || t.tc_bwd_saved == 1) && (t.tc_fwd_split == 0 || t.tc_fwd_split == 1) &&
         (t.fp32_ctas == 1 || t.fp32_ctas == 2) && mult32(t.composite_threads, 64, 512) &&
         mult32(t.sampler_threads, 128, 512);
}
static void to_abi(const snk::Tuning &u, bool tuned, snk_tuning *t) {
  memset(t, 0, sizeof(*t));
  t->tc_fwd_ctas = u.tc_fwd_ctas;
  t->tc_fwd_levels = u.tc_fwd_levels;
  t->tc_fwd_split = u.tc_fwd_split;
  t->fp32_ctas = u.fp32_ctas;
  t->tc_bwd_saved = u.tc_bwd_saved;
  t->composite_threads = u.composite_threads;
  t->sampler_threads = u.sampler_threads;
  t->tuned = tuned ? 1 : 0;
}

int snk_get_tuning(snk_ctx *ctx, snk_tuning *out) {
  if (!ctx || !out) return SNK_ERR_INVALID_ARG;
  to_abi(ctx->tune, ctx->tuned, out);
  return SNK_OK;
}

int snk_set_tuning(snk_ctx *ctx, const snk_tuning *in) {
  if (!ctx || !in) return SNK_ERR_INVALID_ARG;
  if (!tuning_ok(*in)) return fail(ctx, SNK_ERR_INVALID_ARG, "snk_set_tuning: value out of range");
  ctx->tune.tc_fwd_ctas = in->tc_fwd_ctas;
  ctx->tune.tc_fwd_levels = in->tc_fwd_levels;
  ctx->tune.tc_fwd_split = in->tc_fwd_split;
  ctx->tune.fp32_ctas = in->fp32_ctas;
  ctx->tune.tc_bwd_saved = in->tc_bwd_saved;
  ctx->tune.composite_threads = in->composite_threads;
  ctx->tune.sampler_threads = in->sampler_threads;
  ctx->tuned = false;
  return SNK_OK;
}

int snk_autotune(snk_ctx *ctx, const snk_model *model, const snk_window *win, const uint32_t *pix, int B,
                 const snk_sampler *sampler, const snk_params *p, snk_stream_t stream, snk_tuning *out) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  WinParams wp;
  if ((rc = check_window(sink(ctx), win, model->n_slots, &wp))) return rc;
  SamplerParams sp;
  if ((rc = check_sampler(sink(ctx), sampler, &sp))) return rc;
  sp.render = 0;
  if ((rc = check_params(ctx, model, p, false))) return rc;
  if (!pix || B < 1 || B > (1 << 22)) return fail(ctx, SNK_ERR_INVALID_ARG, "need pix and 1 <= B <= 2^22");
  if (ctx->n_views < 1) return fail(ctx, SNK_ERR_INVALID_ARG, "no views: call snk_set_views first");
  if ((rc = ensure_ws(ctx, B, max_samples_for(win, sampler, B)))) return rc;
  const cudaStream_t st = (cudaStream_t)stream;
  // scratch: a per-step state, a gradient accumulator and a render output (the caller's are untouched)
  void *scratch = nullptr;
  const size_t grad_bytes = sizeof(float) * (size_t)lay.n_params;
  const size_t bytes = sizeof(snk_state) + 256 + grad_bytes + 256 + sizeof(float) * 5 * (size_t)B;
  if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SNK_ERR_OOM, "snk_autotune: scratch of %zu bytes could not be allocated", bytes);
  }
  snk_state *state = reinterpret_cast<snk_state *>(scratch);
  float *grads = reinterpret_cast<float *>(static_cast<char *>(scratch) + (sizeof(snk_state) + 255) / 256 * 256);
  float *rout = grads + (grad_bytes + 255) / 256 * 64;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const snk::Tuning saved = ctx->tune;
  snk_params ps = *p;
  ps.grads = grads;
  rc = SNK_OK;
  auto cuda_ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == SNK_OK) rc = fail(ctx, SNK_ERR_CUDA, "snk_autotune: %s", cudaGetErrorString(e));
    return rc == SNK_OK;
  };
  // mean time of reps runs after one warm-up run; <0 on failure
  auto time = [&](auto &&run, int reps) -> double {
    if (run() != SNK_OK) return -1.0;
    if (!cuda_ok(cudaEventRecord(e0, st))) return -1.0;
    for (int i = 0; i < reps; ++i)
      if (run() != SNK_OK) return -1.0;
    if (!cuda_ok(cudaEventRecord(e1, st)) || !cuda_ok(cudaEventSynchronize(e1))) return -1.0;
    float ms = 0.f;
    if (!cuda_ok(cudaEventElapsedTime(&ms, e0, e1))) return -1.0;
    return ms / reps;
  };
  auto sample = [&]() -> int {
    if (launch_sample_segments(ctx->d_views, ctx->n_views, wp, sp, pix, B, 0, step_rays(ctx, model), ctx->cap_samples, state, st,
                               ctx->tune) != cudaSuccess)
      return fail(ctx, SNK_ERR_CUDA, "snk_autotune: sampling failed");
    return SNK_OK;
  };
  uint16_t *tune_acts = nullptr;  // the stored-activation buffer while the stored mode is timed
  auto field = [&](int mode) {
    return run_field(ctx, model, md, &ps, state, mode, st, B, ctx->tune.tc_bwd_saved ? tune_acts : nullptr);
  };
  CompositeArgs ca{};
  ca.sigma_rgb = ctx->sigma_rgb;
  ca.smp_t = ctx->rb.smp_t;
  ca.smp_dt = ctx->rb.smp_dt;
  ca.seg_n = ctx->rb.seg_n;
  ca.seg_off = ctx->rb.seg_off;
  ca.B = B;
  ca.out = rout;
  ca.state = state;
  auto composite = [&]() -> int {
    if (launch_composite(ca, st, ctx->tune) != cudaSuccess) return fail(ctx, SNK_ERR_CUDA, "snk_autotune: composite failed");
    return SNK_OK;
  };
  do {
    if (!cuda_ok(cudaEventCreate(&e0)) || !cuda_ok(cudaEventCreate(&e1))) break;
    if (!cuda_ok(cudaMemsetAsync(state, 0, sizeof(snk_state), st))) break;
    if (!cuda_ok(cudaMemsetAsync(ctx->dsr, 0, sizeof(float) * 4 * (size_t)ctx->cap_samples, st))) break;
    // rays, segments and samples: threads per block
    double best = -1.0;
    int pick = saved.sampler_threads;
    for (int nt : {128, 256, 512}) {
      ctx->tune.sampler_threads = nt;
      const double ms = time(sample, 2);
      if (ms < 0) break;
      if (best < 0 || ms < best) best = ms, pick = nt;
    }
    if (rc) break;
    ctx->tune.sampler_threads = pick;
    if (sample() != SNK_OK) break;  // leave this batch's samples in the workspace
    // field kernels
    if (model->precision != SNK_FP32) {
      // per backward mode (stored activations when their buffer can be had, recompute): the
      // fastest forward shape, then forward + backward decide between the modes
      double best_step = -1.0;
      snk::Tuning pick = ctx->tune;
      for (int sv : {1, 0}) {
        if (sv == 1 && (tune_acts = acts_or_recompute(ctx, model, st)) == nullptr) continue;  // no room: recompute only
        ctx->tune.tc_bwd_saved = sv;
        best = -1.0;
        int pc = saved.tc_fwd_ctas, pl = saved.tc_fwd_levels, ps = saved.tc_fwd_split;
        // (split, CTAs per SM, levels): dedicated gather warps run two CTAs per SM
        const int shapes[8][3] = {{1, 2, 1}, {1, 2, 2}, {0, 1, 1}, {0, 1, 2}, {0, 2, 1}, {0, 2, 2}, {0, 3, 1}, {0, 3, 2}};
        for (const auto &sh : shapes) {
          // no gather in the E4M3 forward: one shape
          if (model->precision == SNK_MIXED_E4M3 && (sh[0] == 1 || sh[2] == 2)) continue;
          ctx->tune.tc_fwd_split = sh[0];
          ctx->tune.tc_fwd_ctas = sh[1];
          ctx->tune.tc_fwd_levels = sh[2];
          const double ms = time([&] { return field(kForward); }, 2);
          if (ms < 0) break;
          if (best < 0 || ms < best) best = ms, ps = sh[0], pc = sh[1], pl = sh[2];
        }
        if (rc) break;
        ctx->tune.tc_fwd_split = ps;
        ctx->tune.tc_fwd_ctas = pc;
        ctx->tune.tc_fwd_levels = pl;
        if (field(kForward) != SNK_OK) break;  // this mode's forward outputs for its backward
        const double b = time([&] { return field(kBackward); }, 1);
        if (b < 0) break;
        if (best_step < 0 || best + b < best_step) best_step = best + b, pick = ctx->tune;
      }
      if (rc) break;
      ctx->tune = pick;
    } else {
      best = -1.0;
      int pc = saved.fp32_ctas;
      for (int c : {1, 2}) {
        ctx->tune.fp32_ctas = c;
        const double f = time([&] { return field(kForward); }, 1);
        const double b = f < 0 ? -1.0 : time([&] { return field(kBackward); }, 1);
        if (b < 0) break;
        if (best < 0 || f + b < best) best = f + b, pc = c;
      }
      if (rc) break;
      ctx->tune.fp32_ctas = pc;
    }
    if (field(kForward) != SNK_OK) break;
    // compositing: threads per block
    best = -1.0;
    int pt = saved.composite_threads;
    for (int nt : {64, 128, 256, 512}) {
      ctx->tune.composite_threads = nt;
      const double ms = time(composite, 2);
      if (ms < 0) break;
      if (best < 0 || ms < best) best = ms, pt = nt;
    }
    if (rc) break;
    ctx->tune.composite_threads = pt;
  } while (false);
  if (rc == SNK_OK) cuda_ok(cudaStreamSynchronize(st));
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(scratch);
  if (rc != SNK_OK) {
    ctx->tune = saved;
    return rc;
  }
  ctx->tuned = true;
  if (out) to_abi(ctx->tune, true, out);
  return SNK_OK;
}

int snk_build_crops(snk_ctx *ctx, const snk_window *win, int margin, int32_t *tile_rects, int32_t *view_rects,
                    snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (!win) return fail(ctx, SNK_ERR_INVALID_ARG, "window is NULL");
  WinParams wp;
  int rc = check_window(sink(ctx), win, win->nx * win->ny, &wp);
  if (rc) return rc;
  if (!tile_rects || !view_rects || margin < 0 || margin > 4096)
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_build_crops: NULL output or margin outside 0..4096");
  if (ctx->n_views < 1) return fail(ctx, SNK_ERR_INVALID_ARG, "no views: call snk_set_views first");
  CropParams cp;
  cp.tile[0] = win->tile_size[0];
  cp.tile[1] = win->tile_size[1];
  cp.margin = margin;
  SNK_CK(ctx, launch_crops(ctx->d_views, ctx->n_views, wp, cp, tile_rects, view_rects, (cudaStream_t)stream));
  return SNK_OK;
}

int snk_ray_pool(snk_ctx *ctx, const snk_window *win, const int32_t *view_rects, uint32_t *pool, int64_t cap,
                 uint32_t *n_pool, snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (!win) return fail(ctx, SNK_ERR_INVALID_ARG, "window is NULL");
  WinParams wp;
  int rc = check_window(sink(ctx), win, win->nx * win->ny, &wp);
  if (rc) return rc;
  if (!view_rects || !pool || !n_pool || cap < 1 || cap > 0xFFFFFFFFll)
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_ray_pool: NULL buffer or cap outside 1..2^32-1");
  if (ctx->n_views < 1) return fail(ctx, SNK_ERR_INVALID_ARG, "no views: call snk_set_views first");
  // scratch sized by the views' whole images (an upper bound of any crop set)
  int64_t max_pixels = 0;
  for (int v = 0; v < ctx->n_views; ++v) max_pixels += (int64_t)ctx->h_views[v].width * ctx->h_views[v].height;
  const int64_t nc = pool_chunks(max_pixels);
  const size_t need = 256 * 16 + (size_t)nc * 4 + 256 + (size_t)max_pixels;
  if (need > ctx->pool_ws_bytes) {
    if (ctx->pool_ws) {
      SNK_CK(ctx, cudaStreamSynchronize((cudaStream_t)stream));
      SNK_CK(ctx, cudaFree(ctx->pool_ws));
      ctx->pool_ws = nullptr;
      ctx->pool_ws_bytes = 0;
    }
    if (cudaMalloc(&ctx->pool_ws, need) != cudaSuccess) {
      cudaGetLastError();
      ctx->pool_ws = nullptr;
      return fail(ctx, SNK_ERR_OOM, "snk_ray_pool: scratch of %zu bytes could not be allocated", need);
    }
    ctx->pool_ws_bytes = need;
  }
  char *w = static_cast<char *>(ctx->pool_ws);
  int64_t *base = reinterpret_cast<int64_t *>(w);
  uint32_t *chunk = reinterpret_cast<uint32_t *>(w + 256 * 16);
  uint8_t *flags = reinterpret_cast<uint8_t *>(w + 256 * 16 + ((size_t)nc * 4 + 255) / 256 * 256);
  SNK_CK(ctx, launch_ray_pool(ctx->d_views, ctx->n_views, wp, view_rects, base, max_pixels, flags, chunk, pool, cap,
                              n_pool, (cudaStream_t)stream));
  return SNK_OK;
}

int snk_occupancy_update(snk_ctx *ctx, const snk_model *model, const snk_params *p, float *density,
                         uint8_t *occupancy, int R, float decay, float threshold, uint32_t seed, uint32_t step,
                         snk_stream_t stream) {
  snk_layout lay;
  ModelDev md;
  int rc = prepare(ctx, model, &lay, &md);
  if (rc) return rc;
  if ((rc = check_params(ctx, model, p, false))) return rc;
  if (!density || !occupancy || R < 8 || R > 512 || R % 8 != 0)
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_occupancy_update: NULL grid or R not a multiple of 8 in 8..512");
  if (!(decay >= 0.0f && decay <= 1.0f) || !(threshold >= 0.0f) || !std::isfinite(threshold))
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_occupancy_update: need 0 <= decay <= 1 and a finite threshold >= 0");
  const int64_t S = (int64_t)model->n_slots * R * R * R;
  if ((rc = ensure_ws(ctx, ctx->cap_rays > 0 ? ctx->cap_rays : 1, S))) return rc;
  const size_t need = 256 + sizeof(float) * (size_t)occ_partials(model->n_slots, R) + 256;
  if (need > ctx->occ_ws_bytes) {
    if (ctx->occ_ws) {
      SNK_CK(ctx, cudaStreamSynchronize((cudaStream_t)stream));
      SNK_CK(ctx, cudaFree(ctx->occ_ws));
      ctx->occ_ws = nullptr;
      ctx->occ_ws_bytes = 0;
    }
    if (cudaMalloc(&ctx->occ_ws, need) != cudaSuccess) {
      cudaGetLastError();
      ctx->occ_ws = nullptr;
      return fail(ctx, SNK_ERR_OOM, "snk_occupancy_update: scratch of %zu bytes could not be allocated", need);
    }
    ctx->occ_ws_bytes = need;
  }
  snk_state *state = static_cast<snk_state *>(ctx->occ_ws);
  // sigma, the only output used, does not depend on the view direction: every point takes ray 0
  float *partial = reinterpret_cast<float *>(static_cast<char *>(ctx->occ_ws) + 256);
  float *thr = partial + occ_partials(model->n_slots, R);
  const cudaStream_t st = (cudaStream_t)stream;
  SNK_CK(ctx, cudaMemsetAsync(state, 0, sizeof(snk_state), st));
  SNK_CK(ctx, launch_occ_points(model->n_slots, R, seed, step, ctx->rb.smp_xyz, ctx->rb.smp_ray, state, st));
  if ((rc = run_field(ctx, model, md, p, state, kForward, st, 1, nullptr))) return rc;
  SNK_CK(ctx, launch_occ_update(model->n_slots, R, ctx->sigma_rgb, decay, threshold, density, occupancy, partial, thr,
                                st));
  return SNK_OK;
}

int snk_draw_batch(snk_ctx *ctx, const uint32_t *pool, const uint32_t *n_pool, int B, uint32_t seed, uint32_t iteration,
                   uint32_t *pix, snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (!pool || !n_pool || !pix || B < 0 || B > (1 << 22))
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_draw_batch: NULL buffer or B outside 0..2^22");
  SNK_CK(ctx, launch_draw(pool, n_pool, B, seed, iteration, pix, (cudaStream_t)stream));
  return SNK_OK;
}

int snk_quantize_e4m3(snk_ctx *ctx, const float *x, int64_t n, float scale, uint8_t *codes, snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!x || !codes)))
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_quantize_e4m3: NULL buffer or negative n");
  if (!(scale > 0.0f) || !std::isfinite(scale))
    return fail(ctx, SNK_ERR_INVALID_ARG, "snk_quantize_e4m3: scale must be positive and finite");
  SNK_CK(ctx, launch_quantize_e4m3(x, n, scale, codes, (cudaStream_t)stream));
  return SNK_OK;
}

int64_t snk_launch_count(void) { return snk::g_launches.load(); }

int snk_wait_selftest(snk_ctx *ctx, int arrive, snk_state *state, snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (!state) return fail(ctx, SNK_ERR_INVALID_ARG, "snk_wait_selftest: state is NULL");
  SNK_CK(ctx, launch_wait_selftest(arrive, state, (cudaStream_t)stream));
  return SNK_OK;
}

int snk_l2_reduction_probe(snk_ctx *ctx, float *table, int64_t n16, int64_t n_ops, int width, uint32_t seed,
                           snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  if (!table || reinterpret_cast<uintptr_t>(table) % 16 != 0 || n16 < 1 || n16 > 0xFFFFFFFFll || n_ops < 0 ||
      (width != 8 && width != 16))
    return fail(ctx, SNK_ERR_INVALID_ARG,
                "snk_l2_reduction_probe: need a 16-byte aligned table, 1 <= n16 < 2^32, n_ops >= 0, width 8 or 16");
  SNK_CK(ctx, launch_red_probe(table, n16, n_ops, width, seed, ctx->sm_count, (cudaStream_t)stream));
  return SNK_OK;
}

int snk_stage_timing(snk_ctx *ctx, int enable) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  SNK_CK(ctx, cudaDeviceSynchronize());
  ctx->timing = enable != 0;
  ctx->recorded.clear();
  ctx->ev_used = 0;
  return SNK_OK;
}

int snk_stage_times(snk_ctx *ctx, double *ms, int64_t *calls, int n) {
  if (!ctx || !ms || !calls || n < 0) return SNK_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    ms[i] = 0.0;
    calls[i] = 0;
  }
  SNK_CK(ctx, cudaDeviceSynchronize());
  for (auto &r : ctx->recorded) {
    float t = 0.f;
    SNK_CK(ctx, cudaEventElapsedTime(&t, r.second.first, r.second.second));
    if (r.first < n) {
      ms[r.first] += t;
      calls[r.first] += 1;
    }
  }
  return SNK_OK;
}

int snk_sync_status(snk_ctx *ctx, const snk_state *state, snk_stream_t stream) {
  if (!ctx || !state) return SNK_ERR_INVALID_ARG;
  SNK_CK(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  uint32_t status = 0;
  SNK_CK(ctx, cudaMemcpy(&status, &state->status, sizeof(status), cudaMemcpyDeviceToHost));
  if (status & kStatusCheck) return fail(ctx, SNK_ERR_DEVICE_CHECK, "a device-side check failed (status %u)", status);
  if (status & kStatusTimeout) return fail(ctx, SNK_ERR_TIMEOUT, "a bounded device wait gave up (status %u)", status);
  if (status & kStatusOverflow) return fail(ctx, SNK_ERR_OVERFLOW, "a step was skipped on non-finite gradients");
  return SNK_OK;
}

}  // extern "C"
