"""Target images of the synthetic scenes (oracle, FP64).  Test infrastructure only.

The paper trains on real WorldView-3 images (Sec. 5.1), not available here.
Stand-in: a heightfield surface z = h(x, y) seen by the synthetic cameras,
either a sum of sinusoids (synth.heightfield) or raster blocks
(synth.blocks).  The colour of a pixel is the Lambertian shading of the
first surface point its ray hits:
    colour = albedo(x, y) * (0.2 + 0.8 max(0, n . s))
with s the sun direction, albedo the bilinear interpolation of the 32 x 32
colour noise over the scene's xy box, and n the unit normal: for the
sinusoids (-dh/dx, -dh/dy, 1)/|.|; for the blocks (0, 0, 1) on a roof, and on
a wall (the hit lies below the roof of the cell entered, coming from another
cell) the horizontal axis across which the ray entered, pointing back out
(the x axis when both changed).  The hit is found by marching the ray from z_max in steps of at most
`step` metres of height and refining the first sign change of
z(t) - h(x(t), y(t)) by bisection to 1e-9 m.  Rays that reach z_min or leave
the box without a hit get colour 0.
"""
import numpy as np

from synth import Blocks, pack_pixel
from .camera import rays_fp64


def _cell(hf, x, y):
    n = hf.H.shape[0]
    j = np.clip(np.floor((x - hf.lo[0]) / (hf.hi[0] - hf.lo[0]) * n), 0, n - 1).astype(np.int64)
    i = np.clip(np.floor((y - hf.lo[1]) / (hf.hi[1] - hf.lo[1]) * n), 0, n - 1).astype(np.int64)
    return i, j


def height(hf, x, y):
    if isinstance(hf, Blocks):
        i, j = _cell(hf, x, y)
        return hf.H[i, j]
    z = np.full_like(x, hf.z_base)
    for a, k, p in zip(hf.amp, hf.k, hf.phase):
        z = z + a * np.sin(2 * np.pi * (k[0] * x + k[1] * y) + p)
    return z


def height_grad(hf, x, y):
    gx = np.zeros_like(x)
    gy = np.zeros_like(y)
    for a, k, p in zip(hf.amp, hf.k, hf.phase):
        c = a * 2 * np.pi * np.cos(2 * np.pi * (k[0] * x + k[1] * y) + p)
        gx = gx + c * k[0]
        gy = gy + c * k[1]
    return gx, gy


def normals(hf, p_out, p_in):
    """Unit normals at hits bracketed by p_out (above the surface) and p_in
    (below it, the shaded point)."""
    if isinstance(hf, Blocks):
        io, jo = _cell(hf, p_out[:, 0], p_out[:, 1])
        ii, ji = _cell(hf, p_in[:, 0], p_in[:, 1])
        wall = ((io != ii) | (jo != ji)) & (hf.H[ii, ji] - p_in[:, 2] > 1e-6)
        nrm = np.zeros_like(p_in)
        nrm[:, 2] = 1.0
        wx = wall & (jo != ji)
        wy = wall & (jo == ji)
        nrm[wx] = 0.0
        nrm[wx, 0] = np.sign(p_out[wx, 0] - p_in[wx, 0])
        nrm[wy] = 0.0
        nrm[wy, 1] = np.sign(p_out[wy, 1] - p_in[wy, 1])
        return nrm
    gx, gy = height_grad(hf, p_in[:, 0], p_in[:, 1])
    nrm = np.stack([-gx, -gy, np.ones_like(gx)], 1)
    return nrm / np.linalg.norm(nrm, axis=1, keepdims=True)


def albedo(hf, x, y):
    g = hf.albedo.shape[0]
    u = np.clip((x - hf.lo[0]) / (hf.hi[0] - hf.lo[0]), 0, 1) * (g - 1)
    v = np.clip((y - hf.lo[1]) / (hf.hi[1] - hf.lo[1]), 0, 1) * (g - 1)
    i0 = np.minimum(np.floor(v).astype(int), g - 2)
    j0 = np.minimum(np.floor(u).astype(int), g - 2)
    fv = (v - i0)[:, None]
    fu = (u - j0)[:, None]
    A = hf.albedo
    return (A[i0, j0] * (1 - fv) * (1 - fu) + A[i0 + 1, j0] * fv * (1 - fu)
            + A[i0, j0 + 1] * (1 - fv) * fu + A[i0 + 1, j0 + 1] * fv * fu)


def _first_hit(hf, top, d, step):
    """March each ray from `top` in steps of about `step` metres of height to the
    first sign change of z - height, then bisect to 1e-9 m.  Returns (found mask,
    lo, hi) with the hit bracketed in [lo, hi] for the found rays."""
    n = top.shape[0]
    z_len = hf.hi[2] - hf.lo[2]
    t_max = z_len / np.maximum(-d[:, 2], 1e-12)
    n_steps = int(np.ceil(z_len / step))
    f_prev = top[:, 2] - height(hf, top[:, 0], top[:, 1])
    t_prev = np.zeros(n)
    hit_lo = np.full(n, np.nan)
    hit_hi = np.full(n, np.nan)
    found = f_prev <= 0
    hit_lo[found] = 0.0
    hit_hi[found] = 0.0
    for k in range(1, n_steps + 1):
        t = t_max * (k / n_steps)
        p = top + t[:, None] * d
        f = p[:, 2] - height(hf, p[:, 0], p[:, 1])
        new = (~found) & (f <= 0)
        hit_lo[new] = t_prev[new]
        hit_hi[new] = t[new]
        found |= new
        t_prev = t
    lo = hit_lo[found]
    hi = hit_hi[found]
    tp = top[found]
    dd = d[found]
    for _ in range(200):
        if lo.size == 0 or np.max(hi - lo) <= 1e-9:
            break
        mid = 0.5 * (lo + hi)
        p = tp + mid[:, None] * dd
        f = p[:, 2] - height(hf, p[:, 0], p[:, 1])
        below = f <= 0
        hi = np.where(below, mid, hi)
        lo = np.where(below, lo, mid)
    return found, lo, hi


def surface_t(hf, top, d, step=1.0):
    """Distance (n,) from `top` along d to the first surface hit inside the box, NaN
    for rays that miss (the depth a perfect model renders with opacity 1)."""
    found, lo, hi = _first_hit(hf, top, d, step)
    t = np.full(top.shape[0], np.nan)
    if lo.size:
        p = top[found] + hi[:, None] * d[found]
        inside = ((p[:, 0] >= hf.lo[0]) & (p[:, 0] <= hf.hi[0]) & (p[:, 1] >= hf.lo[1]) & (p[:, 1] <= hf.hi[1]))
        t[np.flatnonzero(found)[inside]] = hi[inside]
    return t


def shade_rays(hf, top, d, step=1.0):
    """Colour (n, 3) of rays starting at `top` (scene coordinates, z = z_max)
    with unit directions d, against heightfield hf inside its box."""
    n = top.shape[0]
    found, lo, hi = _first_hit(hf, top, d, step)
    tp = top[found]
    dd = d[found]
    out = np.zeros((n, 3))
    if lo.size:
        p = tp + hi[:, None] * dd
        inside = ((p[:, 0] >= hf.lo[0]) & (p[:, 0] <= hf.hi[0]) & (p[:, 1] >= hf.lo[1]) & (p[:, 1] <= hf.hi[1]))
        nrm = normals(hf, tp + lo[:, None] * dd, p)
        lam = 0.2 + 0.8 * np.maximum(0.0, nrm @ hf.sun)
        col = albedo(hf, p[:, 0], p[:, 1]) * lam[:, None]
        out[np.flatnonzero(found)] = np.where(inside[:, None], col, 0.0)
    return out


def render_targets(hf, cameras, step=1.0):
    """Float32 crop images (h, w, 3), one per camera."""
    imgs = []
    for vi, cam in enumerate(cameras):
        r0, c0, h, w = cam.crop
        rr, cc = np.meshgrid(np.arange(r0, r0 + h), np.arange(c0, c0 + w), indexing="ij")
        pix = pack_pixel(np.full(rr.size, vi), rr.ravel(), cc.ravel())
        o, d = rays_fp64(cameras, pix, np.zeros(3), hf.lo[2], hf.hi[2])
        col = shade_rays(hf, o, d, step)
        imgs.append(col.reshape(h, w, 3).astype(np.float32))
    return imgs
