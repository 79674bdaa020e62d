"""Image crops from ground tiles, the ray pool of a window and batch draws
from it (oracle, FP64).  Test infrastructure only.

Sec. 4.3: with the camera model, every image gets, for each 3D tile, a crop
that contains the projections of the tile's 8 corners (a margin around it
in the configurations).  A crop is the pixel rectangle rows
[floor(min row) - margin, ceil(max row) + margin) (columns alike) of the
corners' continuous pixel coordinates, clipped to the image; a view's crop of
a window is the bounding rectangle of its tiles' crops.

Projection: the pixel coordinates (row, col) with localise(row, col, h) =
(x, y).  For the affine camera it is the solution of a 2 x 2 linear system;
for the cubic rational views it is found here by Newton's method with a
central-difference Jacobian, iterated until the step is below 1e-13 pixel
(the definition is the exact root; the iteration only reaches it).

Ray pool (Sec. 4.4): the pixels of the view crops, in (view, row, col)
order, whose rays the window accepts.  A batch draws B of them with the
counter-based generator: word i % 4 of Philox-4x32-10 at counter (i / 4, 0,
0, 0), key (seed, iteration) (stream 0, the ray pick), index = (x >> 8) *
n >> 24.
"""
import math

import numpy as np

from synth import CAM_AFFINE, pack_pixel
from . import camera, philox, sampler


def project(cam, x, y, h):
    """Continuous pixel coordinates (row, col) of ground points (x, y) at height h."""
    x, y, h = (np.atleast_1d(np.asarray(a, np.float64)) for a in (x, y, h))
    if cam.kind == CAM_AFFINE:
        a, b = cam.a, cam.b
        A = np.array([[a[1], a[2]], [b[1], b[2]]])  # d(x, y) / d(col, row)
        rhs = np.stack([x - a[0] - a[3] * h, y - b[0] - b[3] * h])
        col, row = np.linalg.solve(A, rhs)
        return row, col
    row = np.full(x.shape, cam.height / 2.0)
    col = np.full(x.shape, cam.width / 2.0)
    eps = 1e-3
    for _ in range(60):
        x0, y0 = camera.localise(cam, row, col, h)
        xr1, yr1 = camera.localise(cam, row + eps, col, h)
        xr0, yr0 = camera.localise(cam, row - eps, col, h)
        xc1, yc1 = camera.localise(cam, row, col + eps, h)
        xc0, yc0 = camera.localise(cam, row, col - eps, h)
        j00, j01 = (xc1 - xc0) / (2 * eps), (xr1 - xr0) / (2 * eps)
        j10, j11 = (yc1 - yc0) / (2 * eps), (yr1 - yr0) / (2 * eps)
        det = j00 * j11 - j01 * j10
        ex, ey = x - x0, y - y0
        dcol = (j11 * ex - j01 * ey) / det
        drow = (j00 * ey - j10 * ex) / det
        col, row = col + dcol, row + drow
        if np.max(np.abs(dcol)) < 1e-13 and np.max(np.abs(drow)) < 1e-13:
            break
    return row, col


def tile_corners(win, ix, iy):
    """The 8 corners (x, y, h) of window tile (ix, iy)."""
    out = []
    for c in range(8):
        x = win.origin[0] + win.tile_size[0] * (ix + (c & 1))
        y = win.origin[1] + win.tile_size[1] * (iy + ((c >> 1) & 1))
        h = win.origin[2] + (win.tile_size[2] if c & 4 else 0.0)
        out.append((x, y, h))
    return np.array(out)


def crops(cameras, win, margin):
    """tile_rects [n_views][4] lists of (r0, c0, h, w) (window tile k = iy nx + ix)
    and view_rects [n_views] (the bounding rectangle of the non-empty tile rects),
    plus the continuous corner projections [n_views][k] (8 x 2) for ambiguity checks."""
    tiles, views, proj = [], [], []
    for cam in cameras:
        rects, pr = [], []
        for k in range(win.nx * win.ny):
            ix, iy = k % win.nx, k // win.nx
            p = tile_corners(win, ix, iy)
            row, col = project(cam, p[:, 0], p[:, 1], p[:, 2])
            pr.append(np.stack([row, col], 1))
            r0 = min(cam.height, max(0, math.floor(row.min()) - margin))
            c0 = min(cam.width, max(0, math.floor(col.min()) - margin))
            r1 = min(cam.height, max(r0, math.ceil(row.max()) + margin))
            c1 = min(cam.width, max(c0, math.ceil(col.max()) + margin))
            rects.append((r0, c0, r1 - r0, c1 - c0))
        live = [r for r in rects if r[2] > 0 and r[3] > 0]
        if live:
            r0 = min(r[0] for r in live)
            c0 = min(r[1] for r in live)
            views.append((r0, c0, max(r[0] + r[2] for r in live) - r0, max(r[1] + r[3] for r in live) - c0))
        else:
            views.append((0, 0, 0, 0))
        tiles.append(rects)
        proj.append(pr)
    return tiles, views, proj


def ray_pool(cameras, win, view_rects):
    """Accepted packed pixels of the view rectangles, in (view, row, col) order."""
    wf = sampler.window_f32(win)
    parts = []
    for v, (r0, c0, h, w) in enumerate(view_rects):
        if h <= 0 or w <= 0:
            continue
        rr, cc = np.meshgrid(np.arange(r0, r0 + h), np.arange(c0, c0 + w), indexing="ij")
        pix = pack_pixel(np.full(rr.size, v), rr.ravel(), cc.ravel())
        o, d = camera.rays(cameras, pix, win.origin, win.origin[2], win.origin[2] + win.tile_size[2])
        ok = sampler.accepted(o, d, wf)[0]
        parts.append(pix[ok])
    return np.concatenate(parts) if parts else np.zeros(0, np.uint32)


def draw(pool, B, seed, iteration):
    """B pixels drawn from the pool (see the module docstring)."""
    n = len(pool)
    i = np.arange(B, dtype=np.uint64)
    words = philox.philox4x32(np.stack([(i >> np.uint64(2)).astype(np.uint32), np.zeros(B, np.uint32),
                                        np.zeros(B, np.uint32), np.zeros(B, np.uint32)], 1),
                              np.array([seed, iteration], np.uint32))
    x = words[np.arange(B), (i & np.uint64(3)).astype(np.int64)].astype(np.uint64)
    idx = ((x >> np.uint64(8)) * np.uint64(n)) >> np.uint64(24)
    return pool[idx.astype(np.int64)]
