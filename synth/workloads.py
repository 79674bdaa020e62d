"""Workload definitions: scene boxes, views, grid and MLP sizes, batch sizes.

The named workloads restate the benchmark configurations of this project
(single tile FP32, single tile full size, 2x2 window) plus small variants that
the FP64 oracle finishes in seconds.  Everything here is sizes and seeded
draws; no step of the method is computed.
"""
from dataclasses import dataclass, field
import numpy as np

from . import (CAM_AFFINE, CAM_RPC3, Window, blocks, heightfield, pushbroom_cameras, random_pixels,
               dirichlet_mix, pack_pixel, glorot_bound)


@dataclass
class Workload:
    name: str
    tile: tuple                 # (Wt, Ht, Z) metres
    nx: int
    ny: int
    n_views: int
    px: int                     # image side in pixels
    cam_kind: int
    off_nadir: tuple
    L: int
    F: int
    log2_T: int
    n_min: int
    n_max: int
    geo_out: int
    colour: bool
    shared_colour: bool
    n_rays: int
    K_ray: int
    K_min: int
    K_max: int
    mixed: bool = False          # FP16 tables + BF16 MLP on tensor cores
    crop_margin: int = 0
    dirichlet: bool = False
    seed: int = 0
    hidden: int = 64
    notes: str = ""
    scene_kind: str = "sines"    # "blocks": raster blocks (synth.blocks) on a raster x raster grid
    raster: int = 512
    first_layer: str = "f16"     # "e4m3": 8-bit first-layer input, per-tensor scale from the batch
    grid: tuple = (0, 0)         # tiles of the whole scene for a snake sweep; (0, 0): the window is the scene
    view_dirs: bool = False      # colour input [embedding | SH of the ray direction, degrees 0..3]

    @property
    def n_slots(self):
        return self.nx * self.ny

    def grid_tiles(self):
        return self.grid if self.grid[0] > 0 else (self.nx, self.ny)

    def scene_box(self):
        gx, gy = self.grid_tiles()
        lo = np.array([0.0, 0.0, 0.0])
        hi = np.array([gx * self.tile[0], gy * self.tile[1], self.tile[2]])
        return lo, hi

    def window(self, pos=(0, 0), slot=(0, 1, 2, 3)):
        """The window whose lower-left tile is tile `pos` of the grid; slot[iy * nx + ix]
        is the parameter slot of the window's tile (ix, iy)."""
        lo, hi = self.scene_box()
        origin = np.array([pos[0] * self.tile[0], pos[1] * self.tile[1], 0.0])
        return Window(origin=origin, tile_size=np.array(self.tile, float), nx=self.nx, ny=self.ny,
                      scene_lo=lo, scene_hi=hi, slot=tuple(slot))


WORKLOADS = {
    # Plain single-tile FP32 step: 256x256x64 m, 8 affine views 128^2, L8 T2^14.
    "tile256_fp32": Workload("tile256_fp32", (256.0, 256.0, 64.0), 1, 1, 8, 128, CAM_AFFINE, (5.0, 30.0),
                             8, 2, 14, 16, 256, 4, False, True, 1024, 64, 64, 64),
    # Single tile, full size: 512x512x96 m, 16 RPC-like views 1024^2, L16 T2^19, 262144 rays x 96.
    "tile512_full": Workload("tile512_full", (512.0, 512.0, 96.0), 1, 1, 16, 1024, CAM_RPC3, (5.0, 30.0),
                             16, 2, 19, 16, 2048, 16, True, True, 262144, 96, 96, 96, mixed=True),
    # 2x2 window of 512x512x96 m tiles, 16 views 2048^2, 524288 rays in a Dirichlet(0.5) mix.
    "window2x2_full": Workload("window2x2_full", (512.0, 512.0, 96.0), 2, 2, 16, 2048, CAM_RPC3, (5.0, 30.0),
                               16, 2, 19, 16, 2048, 16, True, True, 524288, 128, 64, 128, mixed=True,
                               crop_margin=64, dirichlet=True),
    # Mixed-precision stress: the 2x2 window over raster blocks 5-60 m tall on a 512 x 512 grid,
    # off-nadir up to 40 degrees, 256 samples per ray, E4M3 first-layer input.
    "window2x2_fp8": Workload("window2x2_fp8", (512.0, 512.0, 96.0), 2, 2, 16, 2048, CAM_RPC3, (5.0, 40.0),
                              16, 2, 19, 16, 2048, 16, True, True, 524288, 256, 32, 256, mixed=True,
                              crop_margin=64, dirichlet=True, scene_kind="blocks", first_layer="e4m3"),
    # Snake sweep over an 8 x 8 grid of 512 x 512 x 128 m tiles (4096 x 4096 x 128 m scene), 32 RPC-like
    # views at 4096 px, 262144 rays per iteration on the active 2 x 2 window.
    "sweep_grid8": Workload("sweep_grid8", (512.0, 512.0, 128.0), 2, 2, 32, 4096, CAM_RPC3, (5.0, 30.0),
                            16, 2, 19, 16, 2048, 16, True, True, 262144, 128, 64, 128, mixed=True,
                            crop_margin=64, dirichlet=True, grid=(8, 8)),
    # Small cases for the oracle (seconds on a CPU).
    "tiny_tile": Workload("tiny_tile", (64.0, 64.0, 32.0), 1, 1, 4, 48, CAM_AFFINE, (5.0, 30.0),
                          4, 2, 10, 4, 32, 4, False, True, 96, 24, 24, 24),
    "tiny_window": Workload("tiny_window", (48.0, 48.0, 32.0), 2, 2, 6, 64, CAM_RPC3, (10.0, 35.0),
                            4, 2, 11, 4, 48, 16, True, True, 160, 32, 12, 32, crop_margin=4, dirichlet=True),
    "tiny_sweep": Workload("tiny_sweep", (32.0, 32.0, 24.0), 2, 2, 6, 96, CAM_RPC3, (10.0, 30.0),
                           4, 2, 10, 4, 32, 16, True, True, 96, 16, 4, 16, crop_margin=4, dirichlet=True,
                           grid=(3, 3)),
    "tiny_window_vd": Workload("tiny_window_vd", (48.0, 48.0, 32.0), 2, 2, 6, 64, CAM_RPC3, (10.0, 35.0),
                               4, 2, 11, 4, 48, 16, True, True, 160, 32, 12, 32, crop_margin=4, dirichlet=True,
                               view_dirs=True),
    "tiny_window_fp8": Workload("tiny_window_fp8", (48.0, 48.0, 32.0), 2, 2, 6, 64, CAM_RPC3, (10.0, 40.0),
                                4, 2, 11, 4, 48, 16, True, True, 160, 48, 8, 48, mixed=True, crop_margin=4,
                                dirichlet=True, scene_kind="blocks", raster=64, first_layer="e4m3"),
}


def get(name, **overrides):
    import dataclasses
    w = WORKLOADS[name]
    return dataclasses.replace(w, **overrides) if overrides else w


def scene(w):
    lo, hi = w.scene_box()
    if w.scene_kind == "blocks":
        return blocks(w.seed, lo, hi, n=w.raster)
    amp = 20.0 * min(1.0, w.tile[2] / 64.0) if w.tile[2] >= 32 else 8.0
    return heightfield(w.seed, lo, hi, amplitude=amp, min_wavelength=max(8.0, w.tile[0] / 10.0))


def cameras(w):
    lo, hi = w.scene_box()
    return pushbroom_cameras(w.seed + 1, w.n_views, w.px, w.px, lo, hi, off_nadir=w.off_nadir,
                             kind=w.cam_kind)


def tile_crops(w, cams, pos=(0, 0)):
    """Per view and tile of the window at grid position `pos`: pixel rectangle
    (r0, c0, h, w) that contains the image of the tile's 8 corners, widened by
    the crop margin and clipped to the image (the crops of Sec. 4.3, built from
    the affine part of each synthetic camera as it was drawn)."""
    out = []
    for cam in cams:
        A = np.array([[cam.a[1], cam.a[2]], [cam.b[1], cam.b[2]]])
        Ainv = np.linalg.inv(A)
        rects = []
        for iy in range(w.ny):
            for ix in range(w.nx):
                xs = [(pos[0] + ix) * w.tile[0], (pos[0] + ix + 1) * w.tile[0]]
                ys = [(pos[1] + iy) * w.tile[1], (pos[1] + iy + 1) * w.tile[1]]
                rc = []
                for x in xs:
                    for y in ys:
                        for h in (0.0, w.tile[2]):
                            cc, rr = Ainv @ np.array([x - cam.a[0] - cam.a[3] * h, y - cam.b[0] - cam.b[3] * h])
                            rc.append((rr, cc))
                rc = np.array(rc)
                # a window outside the image gets an empty rectangle at the image border
                r0 = int(min(cam.height, max(0, np.floor(rc[:, 0].min()) - w.crop_margin)))
                c0 = int(min(cam.width, max(0, np.floor(rc[:, 1].min()) - w.crop_margin)))
                r1 = int(min(cam.height, np.ceil(rc[:, 0].max()) + w.crop_margin))
                c1 = int(min(cam.width, np.ceil(rc[:, 1].max()) + w.crop_margin))
                rects.append((r0, c0, max(0, r1 - r0), max(0, c1 - c0)))
        out.append(rects)
    return out


def batch(w, cams, seed, n_rays=None, pos=(0, 0)):
    """Packed pixel ids of one random ray batch for the window at grid position
    `pos`.  Without a Dirichlet mix the pixels are uniform over every view's
    crop; with it, n ~ Multinomial(n_rays, p), p ~ Dirichlet(0.5) rays are drawn
    from the crops of each tile of the window."""
    n_rays = w.n_rays if n_rays is None else n_rays
    if not w.dirichlet:
        return random_pixels(seed, n_rays, cams)
    counts, _ = dirichlet_mix(seed, n_rays, w.n_slots)
    crops = tile_crops(w, cams, pos)
    rng = np.random.default_rng(seed + 7919)
    parts = []
    for t, n in enumerate(counts):
        v = rng.integers(0, len(cams), n)
        rects = np.array([crops[vi][t] for vi in v], np.int64).reshape(-1, 4)
        rr = rects[:, 0] + (rng.random(n) * np.maximum(rects[:, 2], 1)).astype(np.int64)
        cc = rects[:, 1] + (rng.random(n) * np.maximum(rects[:, 3], 1)).astype(np.int64)
        rr = np.clip(rr, 0, cams[0].height - 1)
        cc = np.clip(cc, 0, cams[0].width - 1)
        parts.append(pack_pixel(v, rr, cc))
    pix = np.concatenate(parts)
    return pix[rng.permutation(len(pix))]


def init_params(layout_n_params, geo_shapes, col_shapes, n_slots, n_col_blocks, seed):
    """Initial flat parameter vector (float32): tables U(-1e-4, 1e-4) (NGP),
    MLP matrices Glorot-uniform; layout [slots..., colour blocks...]."""
    rng = np.random.default_rng(seed + 104729)
    parts = []
    for _ in range(n_slots):
        parts.append(rng.uniform(-1e-4, 1e-4, layout_n_params))
        for a, b in geo_shapes:
            parts.append(rng.uniform(-1, 1, a * b) * glorot_bound(b, a))
    for _ in range(n_col_blocks):
        for a, b in col_shapes:
            parts.append(rng.uniform(-1, 1, a * b) * glorot_bound(b, a))
    return np.concatenate(parts).astype(np.float32)
