"""Pins of the oracle's sampler variants (oracle/sampler.py), CPU only.

UNIFORM (the NeRF-XL distribution): on a one-tile window it is the segmented
sampler exactly; on a 2x2 window every sample lies in its segment's tile and
the bins cover the ray.  POINTS: the face point between two segments is
sampled twice, the second copy has delta 0, and compositing ignores its
density -- the paper's remark on N_2 (Sec. 4.5)."""
import numpy as np
import pytest

from synth import workloads as W
from oracle import camera, render, sampler as S, step as OS


def _rays(name, n):
    w = W.get(name, n_rays=n)
    cams = W.cameras(w)
    win = w.window()
    pix = W.batch(w, cams, 5)
    o, d = camera.rays(cams, pix, win.origin, win.origin[2], win.origin[2] + win.tile_size[2])
    return w, S.window_f32(win), o, d


def test_uniform_on_one_tile_is_the_segmented_sampler():
    w, wf, o, d = _rays("tiny_tile", 64)
    assert w.K_min <= w.K_ray <= w.K_max
    for render in (False, True):
        seg = S.segments(o, d, wf, w.K_ray, w.K_min, w.K_max)
        smp = S.stratified(o, d, seg, wf, 3, 1, render=render)
        seg_u = S.segments_uniform(o, d, wf, w.K_ray, 3, 1, render=render)
        smp_u = S.stratified(o, d, seg_u, wf, 3, 1, render=render, mode=S.UNIFORM)
        for f in ("slot", "t0", "t1", "K", "ray_off"):
            assert np.array_equal(getattr(seg_u, f), getattr(seg, f)), f
        assert np.array_equal(smp_u.t, smp.t) and np.array_equal(smp_u.dt, smp.dt)
        assert np.array_equal(smp_u.xyz, smp.xyz)


def test_uniform_samples_lie_in_their_tiles_and_cover_the_ray():
    w, wf, o, d = _rays("tiny_window", 200)
    seg = S.segments_uniform(o, d, wf, w.K_ray, 3, 1)
    smp = S.stratified(o, d, seg, wf, 3, 1, mode=S.UNIFORM)
    crossing = 0
    for i in np.flatnonzero(seg.ray_ok):
        sl = slice(seg.ray_off[i], seg.ray_off[i + 1])
        assert seg.ray_off[i + 1] - seg.ray_off[i] == w.K_ray
        t = smp.t[sl].astype(np.float64)
        assert np.all(np.diff(t) > 0)
        assert abs(smp.dt[sl].astype(np.float64).sum() - (seg.t_out[i] - seg.t_in[i])) <= 1e-5 * (seg.t_out[i])
        p = o[i].astype(np.float64) + t[:, None] * d[i].astype(np.float64)
        tiles = [wf.slot.index(int(k)) for s in range(seg.n_seg[i]) for k in [seg.slot[i, s]] * int(seg.K[i, s])]
        ix, iy = np.array(tiles) % wf.nx, np.array(tiles) // wf.nx
        eps = 1e-4
        assert np.all((ix == 0) | (p[:, 0] >= wf.split[0] - eps)) and np.all((ix == 1) | (p[:, 0] <= wf.split[0] + eps))
        assert np.all((iy == 0) | (p[:, 1] >= wf.split[1] - eps)) and np.all((iy == 1) | (p[:, 1] <= wf.split[1] + eps))
        crossing += seg.n_seg[i] > 1
    assert crossing > 10


def test_points_sample_the_face_twice_and_ignore_the_second_copy():
    w, wf, o, d = _rays("tiny_window", 200)
    seg = S.segments(o, d, wf, w.K_ray, w.K_min, w.K_max)
    smp = S.stratified(o, d, seg, wf, 3, 1, mode=S.POINTS)
    rng = np.random.default_rng(0)
    sigma = rng.uniform(0.0, 0.5, len(smp.t))
    rgb = rng.uniform(0, 1, (len(smp.t), 3))
    want = render.composite(sigma, rgb, smp.t.astype(np.float64), smp.dt.astype(np.float64), seg.ray_off)
    faces = 0
    sigma2 = sigma.copy()
    for i in np.flatnonzero(seg.n_seg > 1):
        p = seg.ray_off[i]
        assert smp.dt[p] == 0  # the ray's first point carries no interval
        for s in range(1, seg.n_seg[i]):
            p += int(seg.K[i, s - 1])
            assert smp.t[p] == smp.t[p - 1] == seg.t1[i, s - 1] == seg.t0[i, s]  # F_{s} and N_{s+1}
            assert smp.dt[p] == 0
            sigma2[p] = 1e3  # the N_{s+1} density: ignored
            faces += 1
        sl = slice(seg.ray_off[i], seg.ray_off[i + 1])
        assert abs(smp.dt[sl].astype(np.float64).sum() - (seg.t_out[i] - seg.t_in[i])) <= 1e-5 * seg.t_out[i]
    assert faces > 10
    got = render.composite(sigma2, rgb, smp.t.astype(np.float64), smp.dt.astype(np.float64), seg.ray_off)
    for a, b in zip(got[:3], want[:3]):
        assert np.array_equal(a, b)
