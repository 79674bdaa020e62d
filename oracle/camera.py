"""Satellite camera localisation and on-the-fly rays (oracle, FP64).
Test infrastructure only.

Paper basis: rays are computed on the fly from each image's RPC camera model
instead of being stored (Sec. 3, "1.4TB" remark; Sec. 4.6, "On-the-fly Ray
Calculation"), and coordinates are moved to a local frame before sampling
(Sec. 4.2).  The paper does not define the ray; reading (the Sat-NeRF /
SAT-NGP convention): localise the pixel centre at the top (z_max) and bottom
(z_min) of the scene, the ray is the line through the two points, starting at
the top point.

Arithmetic is a fixed sequence of IEEE binary64 operations (no fused
multiply-add), written out here in that sequence; rounding to binary32 happens
only on the final window-local origin and unit direction.
"""
import numpy as np

from synth import CAM_AFFINE, CAM_RPC3, RPC_MONOMIALS, unpack_pixel


def _poly(coef, c, r, h):
    """sum_i coef[i] * m_i(c, r, h), monomials in RPC_MONOMIALS order, summed
    left to right; each monomial is the left-to-right product of its factors."""
    vals = {"c": c, "r": r, "h": h}
    acc = None
    for i, fac in enumerate(RPC_MONOMIALS):
        if len(fac) == 0:
            term = np.full_like(c, coef[i])
        else:
            m = vals[fac[0]]
            for f in fac[1:]:
                m = m * vals[f]
            term = coef[i] * m
        acc = term if acc is None else acc + term
    return acc


def localise(cam, row, col, h):
    """Ground (x, y) in scene metres of image point (row, col) (continuous pixel
    coordinates) at height h, float64 arrays."""
    row = np.asarray(row, np.float64)
    col = np.asarray(col, np.float64)
    h = np.broadcast_to(np.asarray(h, np.float64), row.shape).astype(np.float64)
    if cam.kind == CAM_AFFINE:
        a, b = cam.a, cam.b
        x = ((a[0] + a[1] * col) + a[2] * row) + a[3] * h
        y = ((b[0] + b[1] * col) + b[2] * row) + b[3] * h
        return x, y
    if cam.kind != CAM_RPC3:
        raise ValueError("unknown camera kind")
    rn = (row - cam.off[0]) / cam.scale[0]
    cn = (col - cam.off[1]) / cam.scale[1]
    hn = (h - cam.off[2]) / cam.scale[2]
    x = cam.off[3] + cam.scale[3] * (_poly(cam.coef[0], cn, rn, hn) / _poly(cam.coef[1], cn, rn, hn))
    y = cam.off[4] + cam.scale[4] * (_poly(cam.coef[2], cn, rn, hn) / _poly(cam.coef[3], cn, rn, hn))
    return x, y


def rays_fp64(cameras, pix, window_origin, z_min, z_max):
    """FP64 ray of each packed pixel id: origin = top point (z = z_max) minus the
    window origin, direction = unit vector from the top point to the bottom point
    (z = z_min).  Returns (o, d) float64 (n, 3) before rounding."""
    v, r, c = unpack_pixel(pix)
    n = len(v)
    top = np.zeros((n, 3))
    bot = np.zeros((n, 3))
    for vi in np.unique(v):
        m = v == vi
        cam = cameras[vi]
        rr = r[m].astype(np.float64) + 0.5
        cc = c[m].astype(np.float64) + 0.5
        xt, yt = localise(cam, rr, cc, z_max)
        xb, yb = localise(cam, rr, cc, z_min)
        top[m] = np.stack([xt, yt, np.full_like(xt, z_max)], 1)
        bot[m] = np.stack([xb, yb, np.full_like(xb, z_min)], 1)
    o = top - np.asarray(window_origin, np.float64)[None, :]
    D = bot - top
    norm = np.sqrt((D[:, 0] * D[:, 0] + D[:, 1] * D[:, 1]) + D[:, 2] * D[:, 2])
    d = D / norm[:, None]
    return o, d


def rays(cameras, pix, window_origin, z_min, z_max):
    """Window-local binary32 rays (o, d), each (n, 3) float32: the FP64 values
    rounded to nearest."""
    o, d = rays_fp64(cameras, pix, window_origin, z_min, z_max)
    return o.astype(np.float32), d.astype(np.float32)
