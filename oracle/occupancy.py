"""Occupancy grid of each tile and the culling of samples in empty space
(oracle, FP64 densities, binary32 cell decisions).  Test infrastructure only.

Sec. 4.1: training follows SAT-NGP, which culls the samples that fall in
empty space using a coarse voxel grid.  Reading: each tile (parameter slot)
has an R^3 grid over its unit cube; cell (x, y, z) of a tile-local point l is
min(floor(l R), R - 1) per axis, in binary32, stored at (z R + y) R + x.  The
stratified candidates of a segment are placed as without culling and only the
ones whose cell is occupied become samples, each keeping its bin width as
delta: a culled sample is a sample of zero density, which compositing skips
exactly (its alpha is 0, the transmittance does not change).

Update: every cell of slot k gets sigma at p = (cell + u) x (1 / R) (binary32
per axis, u = words 0..2 of Philox-4x32-10 at counter (cell, k, 3, 0), key
(seed, step), each (w >> 8) 2^-24) with the slot's field; density <- max(decay
x density, sigma); occupied <- density > min(threshold, mean of the slot's
densities).
"""
import numpy as np

from . import philox, sampler

F32 = np.float32


def cells(l, R):
    """Cell index of tile-local points l (S, 3) float32 (binary32 decisions)."""
    c = np.floor((np.asarray(l, F32) * F32(R)).astype(F32)).astype(np.int64)
    c = np.clip(c, 0, R - 1)
    return (c[:, 2] * R + c[:, 1]) * R + c[:, 0]


def points(k, R, seed, step):
    """Update points (R^3, 3) float32 of slot k, in cell order."""
    n = R ** 3
    cell = np.arange(n, dtype=np.uint32)
    w = philox.philox4x32(np.stack([cell, np.full(n, k, np.uint32), np.full(n, 3, np.uint32),
                                    np.zeros(n, np.uint32)], 1), np.array([seed, step], np.uint32))
    c = np.stack([cell % R, (cell // R) % R, cell // (R * R)], 1).astype(F32)
    u = (w[:, :3] >> np.uint32(8)).astype(F32) * F32(2.0 ** -24)
    inv = F32(F32(1.0) / F32(R))
    return ((c + u).astype(F32) * inv).astype(F32)


def update(cfg, flat, density, R, decay, threshold, seed, step):
    """New (density, occupied) of all slots; density (n_slots, R^3) float64."""
    from .step import field_forward
    new = np.array(density, np.float64, copy=True)
    occ = np.zeros(new.shape, bool)
    for k in range(cfg.n_slots):
        p = points(k, R, seed, step)
        smp = sampler.Samples(np.zeros(len(p), np.int64), np.full(len(p), k, np.int64), np.zeros(len(p), F32),
                              np.zeros(len(p), F32), p)
        # sigma does not depend on a view direction; any direction serves the colour input
        sigma, _, _ = field_forward(cfg, flat, smp, dirs=np.array([[0.0, 0.0, -1.0]]))
        new[k] = np.maximum(decay * new[k], sigma)
        occ[k] = new[k] > min(threshold, new[k].mean())
    return new, occ


def cull(seg, smp, occ, R):
    """Keep the samples whose cell of their slot's grid is occupied; returns the
    kept Samples and a copy of seg whose K counts the kept samples per segment
    and whose ray_off is the CSR of the kept samples."""
    keep = occ[smp.slot, cells(smp.xyz, R)] if len(smp.slot) else np.zeros(0, bool)
    # segment of every sample: the non-empty segments of each ray, in order
    seg_id = []
    for i in range(len(seg.ray_ok)):
        for s in range(3):
            if seg.K[i, s] > 0:
                seg_id.append(np.full(int(seg.K[i, s]), i * 3 + s))
    seg_id = np.concatenate(seg_id) if seg_id else np.zeros(0, np.int64)
    K = np.bincount(seg_id[keep], minlength=3 * len(seg.ray_ok)).reshape(-1, 3)
    out = sampler.Segments(seg.ray_ok, seg.t_in, seg.t_out, seg.n_seg, seg.slot, seg.t0, seg.t1, K,
                           np.concatenate([[0], np.cumsum(K.sum(1))]).astype(np.int64))
    kept = sampler.Samples(smp.ray[keep], smp.slot[keep], smp.t[keep], smp.dt[keep], smp.xyz[keep])
    return out, kept
