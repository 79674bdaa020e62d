// Host-side validation of the descriptors that more than one entry point takes (window,
// sampler, camera), and the kernel constants derived from them.  One definition serves the
// context entry points (api.cu) and the allocation-free sampler (noalloc.cu), so both accept
// exactly the same inputs and round the binary64 window to the same binary32 constants: their
// discrete results (acceptance, segment bounds, sample counts) are then identical bit for bit.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "kernels.cuh"

namespace snk {

int ErrSink::operator()(int code, const char *fmt, ...) const {
  if (buf && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, len, fmt, ap);
    va_end(ap);
  }
  return code;
}

int check_window(const ErrSink &fail, const snk_window *w, int n_slots, WinParams *o) {
  if (!w) return fail(SNK_ERR_INVALID_ARG, "window is NULL");
  if ((w->nx != 1 && w->nx != 2) || (w->ny != 1 && w->ny != 2))
    return fail(SNK_ERR_INVALID_ARG, "window nx, ny must be 1 or 2");
  if (w->nx * w->ny != n_slots)
    return fail(SNK_ERR_INVALID_ARG, "window has %d tiles but the model has %d slots", w->nx * w->ny, n_slots);
  int seen = 0;
  for (int q = 0; q < n_slots; ++q) {
    if (w->slot[q] < 0 || w->slot[q] >= n_slots || (seen >> w->slot[q]) & 1)
      return fail(SNK_ERR_INVALID_ARG, "window slot[] must be a permutation of 0..%d", n_slots - 1);
    seen |= 1 << w->slot[q];
  }
  for (int a = 0; a < 3; ++a) {
    if (!(w->tile_size[a] > 0.0)) return fail(SNK_ERR_INVALID_ARG, "tile_size must be positive");
    if (!(w->scene_hi[a] > w->scene_lo[a])) return fail(SNK_ERR_INVALID_ARG, "scene box is empty");
  }
  memset(o, 0, sizeof(*o));
  for (int a = 0; a < 3; ++a) o->origin[a] = w->origin[a];
  o->z_min = w->origin[2];
  o->z_max = w->origin[2] + w->tile_size[2];
  // binary32 window constants: the correctly rounded images of the binary64 descriptor
  o->win_hi[0] = (float)(w->nx * w->tile_size[0]);
  o->win_hi[1] = (float)(w->ny * w->tile_size[1]);
  o->win_hi[2] = (float)w->tile_size[2];
  for (int a = 0; a < 3; ++a) {
    o->scene_lo[a] = (float)(w->scene_lo[a] - w->origin[a]);
    o->scene_hi[a] = (float)(w->scene_hi[a] - w->origin[a]);
    o->inv_size[a] = (float)(1.0 / w->tile_size[a]);
  }
  o->split[0] = (float)w->tile_size[0];
  o->split[1] = (float)w->tile_size[1];
  o->nx = w->nx;
  o->ny = w->ny;
  for (int q = 0; q < 4; ++q) o->slot[q] = q < n_slots ? w->slot[q] : 0;
  o->n_slots = n_slots;
  return SNK_OK;
}

int check_sampler(const ErrSink &fail, const snk_sampler *s, SamplerParams *o) {
  if (!s) return fail(SNK_ERR_INVALID_ARG, "sampler is NULL");
  if (s->K_min < 1 || s->K_max < s->K_min || s->K_max > 4096 || s->K_ray < 1 || s->K_ray > 4096)
    return fail(SNK_ERR_INVALID_ARG, "need 1 <= K_min <= K_max <= 4096 and 1 <= K_ray <= 4096");
  if (s->occ_res < 0 || s->occ_res > 1024 || (s->occ_res > 0) != (s->occupancy != nullptr))
    return fail(SNK_ERR_INVALID_ARG, "occupancy: need 1 <= occ_res <= 1024 with a grid, or occ_res 0 without");
  if (s->mode != SNK_SAMPLE_SEGMENTS && s->mode != SNK_SAMPLE_UNIFORM && s->mode != SNK_SAMPLE_POINTS)
    return fail(SNK_ERR_INVALID_ARG, "sampler mode must be SNK_SAMPLE_SEGMENTS, _UNIFORM or _POINTS");
  if (s->mode != SNK_SAMPLE_SEGMENTS && s->occ_res > 0)
    return fail(SNK_ERR_INVALID_ARG, "occupancy culling needs SNK_SAMPLE_SEGMENTS");
  if (s->mode == SNK_SAMPLE_POINTS && s->K_min < 2)
    return fail(SNK_ERR_INVALID_ARG, "SNK_SAMPLE_POINTS needs K_min >= 2 (both segment ends)");
  memset(o, 0, sizeof(*o));
  o->K_ray = s->K_ray;
  o->K_min = s->K_min;
  o->K_max = s->K_max;
  o->render = s->render ? 1 : 0;
  o->seed = s->seed;
  o->iteration = s->iteration;
  o->use_state_iteration = 0;
  o->occ_res = s->occ_res;
  o->occ = s->occ_res > 0 ? s->occupancy : nullptr;
  o->mode = s->mode;
  return SNK_OK;
}

int check_camera(const ErrSink &fail, const snk_camera &c, int v, DevView *d) {
  if (c.kind != SNK_CAM_AFFINE && c.kind != SNK_CAM_RPC3)
    return fail(SNK_ERR_INVALID_ARG, "camera %d: unknown kind %d", v, c.kind);
  if (c.crop_h < 0 || c.crop_w < 0 || c.crop_r0 < 0 || c.crop_c0 < 0 || c.crop_r0 + c.crop_h > 4096 ||
      c.crop_c0 + c.crop_w > 4096)
    return fail(SNK_ERR_INVALID_ARG, "camera %d: crop outside 0..4095", v);
  if (c.kind == SNK_CAM_RPC3)
    for (int q = 0; q < 3; ++q)
      if (c.scale[q] == 0.0) return fail(SNK_ERR_INVALID_ARG, "camera %d: zero normalisation scale", v);
  memset(d, 0, sizeof(*d));
  d->kind = c.kind;
  d->width = c.width;
  d->height = c.height;
  d->crop_r0 = c.crop_r0;
  d->crop_c0 = c.crop_c0;
  d->crop_h = c.crop_h;
  d->crop_w = c.crop_w;
  memcpy(d->a, c.a, sizeof(d->a));
  memcpy(d->b, c.b, sizeof(d->b));
  memcpy(d->off, c.off, sizeof(d->off));
  memcpy(d->scale, c.scale, sizeof(d->scale));
  memcpy(d->coef, c.coef, sizeof(d->coef));
  d->crop = nullptr;
  return SNK_OK;
}

}  // namespace snk
