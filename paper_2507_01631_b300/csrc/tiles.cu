// Tile residency for the snake sweep (Sec. 4.4): only the tiles of the active
// 2x2 window live in a model's slots; every other tile's trainable state is
// parked elsewhere -- pinned host memory, or device staging for copies that
// overlap training -- and brought back when the window reaches it.
//
// A parked tile is one contiguous block (offsets rounded up to 256 bytes):
//   [params: tile_params x f32 | m: tile_params x f32 | v: tile_params x f32 |
//    params_lp: tile_params x u16 | Adam step count: i32]
// The slot's gradient accumulator is not part of it: it is zero between steps.
// Copies are cudaMemcpyAsync with cudaMemcpyDefault, one per array, so the
// block may be host (pinned, for asynchrony) or device memory.
#include <cstring>

#include "kernels.cuh"

namespace {

int64_t round256(int64_t x) { return (x + 255) / 256 * 256; }

struct TileBlock {
  int64_t n;  // tile_params
  int64_t off_params, off_m, off_v, off_lp, off_step, bytes;
};

TileBlock tile_block(const snk_layout &lay) {
  TileBlock b;
  b.n = lay.tile_params;
  b.off_params = 0;
  b.off_m = round256(b.off_params + 4 * b.n);
  b.off_v = round256(b.off_m + 4 * b.n);
  b.off_lp = round256(b.off_v + 4 * b.n);
  b.off_step = round256(b.off_lp + 2 * b.n);
  b.bytes = round256(b.off_step + 4);
  return b;
}

// dir 0: slot -> block (park), 1: block -> slot (unpark)
int tile_copy(snk_ctx *ctx, const snk_model *model, const snk_params *p, int slot, void *block, int dir,
              snk_stream_t stream) {
  if (!ctx) return SNK_ERR_INVALID_ARG;
  snk_layout lay;
  int rc = snk_model_layout(model, &lay);
  if (rc != SNK_OK) return rc;
  if (!p || !p->params || !p->adam_m || !p->adam_v || !p->adam_step || !block) return SNK_ERR_INVALID_ARG;
  if (model->precision != SNK_FP32 && !p->params_lp) return SNK_ERR_INVALID_ARG;
  if (slot < 0 || slot >= model->n_slots) return SNK_ERR_INVALID_ARG;
  const TileBlock b = tile_block(lay);
  char *blk = static_cast<char *>(block);
  const int64_t first = (int64_t)slot * lay.tile_params;
  struct Part {
    void *dev;
    int64_t off, bytes;
  };
  const Part parts[5] = {{p->params + first, b.off_params, 4 * b.n},
                         {p->adam_m + first, b.off_m, 4 * b.n},
                         {p->adam_v + first, b.off_v, 4 * b.n},
                         {p->params_lp ? p->params_lp + first : nullptr, b.off_lp, 2 * b.n},
                         {p->adam_step + slot, b.off_step, 4}};
  for (const Part &q : parts) {
    if (!q.dev) continue;
    void *dst = dir == 0 ? static_cast<void *>(blk + q.off) : q.dev;
    const void *src = dir == 0 ? q.dev : static_cast<const void *>(blk + q.off);
    if (cudaMemcpyAsync(dst, src, (size_t)q.bytes, cudaMemcpyDefault, (cudaStream_t)stream) != cudaSuccess) {
      cudaGetLastError();
      return SNK_ERR_CUDA;
    }
  }
  return SNK_OK;
}

}  // namespace

extern "C" {

int snk_tile_bytes(const snk_model *model, int64_t *bytes) {
  snk_layout lay;
  if (!bytes) return SNK_ERR_INVALID_ARG;
  const int rc = snk_model_layout(model, &lay);
  if (rc != SNK_OK) return rc;
  *bytes = tile_block(lay).bytes;
  return SNK_OK;
}

int snk_tile_park(snk_ctx *ctx, const snk_model *model, const snk_params *p, int slot, void *dst,
                  snk_stream_t stream) {
  return tile_copy(ctx, model, p, slot, dst, 0, stream);
}

int snk_tile_unpark(snk_ctx *ctx, const snk_model *model, const snk_params *p, int slot, const void *src,
                    snk_stream_t stream) {
  return tile_copy(ctx, model, p, slot, const_cast<void *>(src), 1, stream);
}

}  // extern "C"
