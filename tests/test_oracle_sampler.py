"""Pins of the oracle's acceptance test and segmented sampler (Sec. 4.4, 4.5):
brute-force marching on tiny inputs, the at-most-3-tiles property, contiguous
segments that meet exactly on tile faces, and delta sums (CPU only)."""
import numpy as np
import pytest

import synth
from synth import workloads as W
from oracle import sampler, camera

F32 = np.float32


def _rays(n, seed, box_hi, spread=0.7):
    """Rays from above a box [0, box_hi] going down at up to ~40 deg off nadir,
    some of them entering through the sides."""
    rng = np.random.default_rng(seed)
    o = np.stack([rng.uniform(-0.2 * box_hi[0], 1.2 * box_hi[0], n),
                  rng.uniform(-0.2 * box_hi[1], 1.2 * box_hi[1], n),
                  np.full(n, box_hi[2])], 1)
    d = np.stack([rng.uniform(-spread, spread, n), rng.uniform(-spread, spread, n), -np.ones(n)], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(F32), d.astype(F32)


def _window(nx, ny, tile, scene_tiles=None, offset=(0, 0)):
    """Window of nx x ny tiles; the scene may be larger (scene_tiles) with the
    window at tile offset `offset`."""
    st = scene_tiles or (nx, ny)
    lo = np.zeros(3)
    hi = np.array([st[0] * tile[0], st[1] * tile[1], tile[2]])
    origin = np.array([offset[0] * tile[0], offset[1] * tile[1], 0.0])
    return synth.Window(origin=origin, tile_size=np.array(tile, float), nx=nx, ny=ny, scene_lo=lo, scene_hi=hi)


def _march_labels(o, d, wf, t_lo, t_hi, n=20001):
    """FP64 march: tile label (0..3) of points in the window box, -1 outside
    the window but inside the scene box, -2 outside the scene box."""
    ts = np.linspace(t_lo, t_hi, n)
    p = o.astype(np.float64)[None, :] + ts[:, None] * d.astype(np.float64)[None, :]
    whi = wf.win_hi.astype(np.float64)
    in_win = np.all((p >= 0) & (p <= whi[None, :]), axis=1)
    in_scene = np.all((p >= wf.scene_lo.astype(np.float64)) & (p <= wf.scene_hi.astype(np.float64)), axis=1)
    ix = (p[:, 0] > wf.split[0]).astype(int) if wf.nx == 2 else np.zeros(n, int)
    iy = (p[:, 1] > wf.split[1]).astype(int) if wf.ny == 2 else np.zeros(n, int)
    lab = np.where(in_win, iy * wf.nx + ix, np.where(in_scene, -1, -2))
    return ts, lab


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 2), (2, 1)])
def test_segments_partition_the_box_interval_brute_force(nx, ny):
    tile = (40.0, 40.0, 30.0)
    win = _window(nx, ny, tile)
    wf = sampler.window_f32(win)
    o, d = _rays(300, 11 + nx + ny, wf.win_hi.astype(np.float64))
    seg = sampler.segments(o, d, wf, 32, 8, 32)
    n_hit = 0
    for i in range(len(o)):
        L = float(np.linalg.norm(wf.win_hi))
        ts, lab = _march_labels(o[i], d[i], wf, -0.5, 1.5 * L)
        inside = lab >= 0
        if not seg.ray_ok[i]:
            assert inside.sum() <= 2, "rejected ray crosses the box"
            continue
        n_hit += 1
        ns = seg.n_seg[i]
        assert 1 <= ns <= 3
        t0, t1 = seg.t0[i, :ns], seg.t1[i, :ns]
        assert np.all(t1 > t0)
        assert np.all(t0[1:] == t1[:-1]), "segments must meet exactly on the tile face"
        assert t0[0] == seg.t_in[i] and t1[-1] == seg.t_out[i]
        # interval = brute-force inside set
        tin_bf, tout_bf = ts[inside][0], ts[inside][-1]
        step = ts[1] - ts[0]
        assert abs(tin_bf - seg.t_in[i]) <= 2 * step and abs(tout_bf - seg.t_out[i]) <= 2 * step
        # every marched point strictly inside a segment carries that segment's tile
        for s in range(ns):
            m = (ts > t0[s] + 2 * step) & (ts < t1[s] - 2 * step)
            if m.any():
                assert np.all(lab[m] == seg.slot[i, s])
        # distinct consecutive tiles
        assert np.all(seg.slot[i, 1:ns] != seg.slot[i, :ns - 1])
    assert n_hit > 100


def test_at_most_three_tiles_and_face_points_shared():
    win = _window(2, 2, (50.0, 50.0, 40.0))
    wf = sampler.window_f32(win)
    o, d = _rays(2000, 5, wf.win_hi.astype(np.float64), spread=0.9)
    seg = sampler.segments(o, d, wf, 64, 4, 64)
    assert seg.n_seg.max() <= 3
    assert (seg.n_seg == 3).sum() > 0 and (seg.n_seg == 2).sum() > 0
    for i in np.flatnonzero(seg.n_seg >= 2):
        for s in range(seg.n_seg[i] - 1):
            tf = seg.t1[i, s]
            p = o[i].astype(np.float64) + float(tf) * d[i].astype(np.float64)
            on_x = abs(p[0] - 50.0) < 1e-4 * 50
            on_y = abs(p[1] - 50.0) < 1e-4 * 50
            assert on_x or on_y, "segment boundary must lie on an interior tile face"


def test_acceptance_rejects_rays_crossing_unloaded_tiles():
    """Window = tiles (1..2, 1..2) of a 4x4-tile scene: accepted iff the ray's
    path inside the scene box stays inside the window (brute force)."""
    tile = (30.0, 30.0, 25.0)
    win = _window(2, 2, tile, scene_tiles=(4, 4), offset=(1, 1))
    wf = sampler.window_f32(win)
    rng = np.random.default_rng(3)
    n = 400
    o = np.stack([rng.uniform(-20, 80, n), rng.uniform(-20, 80, n), np.full(n, 25.0)], 1).astype(F32)
    d = np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.8, 0.8, n), -np.ones(n)], 1)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(F32)
    seg = sampler.segments(o, d, wf, 16, 4, 16)
    n_acc = n_rej_cross = 0
    for i in range(n):
        ts, lab = _march_labels(o[i], d[i], wf, 0.0, 80.0, n=8001)
        in_scene = lab >= -1
        crosses_unloaded = np.any(lab[in_scene] == -1) if in_scene.any() else False
        step = ts[1] - ts[0]
        near_edge = False
        if in_scene.any():
            # skip rays that touch the window boundary within one march step
            idx = np.flatnonzero(in_scene)
            tt = ts[idx]
            p = o[i].astype(np.float64)[None, :] + tt[:, None] * d[i].astype(np.float64)[None, :]
            dist = np.min(np.abs(np.concatenate([p[:, :2], p[:, :2] - wf.win_hi[:2].astype(np.float64)], 1)))
            near_edge = dist < 2 * step
        if near_edge:
            continue
        if seg.ray_ok[i]:
            n_acc += 1
            assert not crosses_unloaded
        elif in_scene.any():
            n_rej_cross += 1
            assert crosses_unloaded
    assert n_acc > 20 and n_rej_cross > 20


def test_single_tile_accepts_every_hitting_ray_and_K_is_K_ray():
    w = W.get("tile256_fp32")
    cams = W.cameras(w)
    pix = W.batch(w, cams, 2)
    o, d = camera.rays(cams, pix, np.zeros(3), 0.0, 64.0)
    wf = sampler.window_f32(w.window())
    seg = sampler.segments(o, d, wf, 64, 64, 64)
    t_in, t_out, _ = sampler.slab(o, d, np.zeros(3, F32), wf.win_hi)
    assert np.array_equal(seg.ray_ok.astype(bool), t_in < t_out)
    assert np.all(seg.n_seg[seg.ray_ok > 0] == 1)
    assert np.all(seg.K[seg.ray_ok > 0, 0] == 64)
    assert seg.ray_off[-1] == 64 * int(seg.ray_ok.sum())


def test_samples_per_segment_rule():
    """K = clamp(rint(K_ray len_seg / len_ray), K_min, K_max), half to even."""
    win = _window(2, 2, (50.0, 50.0, 40.0))
    wf = sampler.window_f32(win)
    o, d = _rays(500, 8, wf.win_hi.astype(np.float64), spread=0.9)
    seg = sampler.segments(o, d, wf, 128, 16, 100)
    for i in np.flatnonzero(seg.ray_ok):
        L = float(seg.t_out[i]) - float(seg.t_in[i])
        for s in range(seg.n_seg[i]):
            frac = (float(seg.t1[i, s]) - float(seg.t0[i, s])) / L
            k = seg.K[i, s]
            assert 16 <= k <= 100
            ideal = 128 * frac
            if 16.5 < ideal < 99.5:
                assert abs(k - ideal) <= 0.5 + 1e-3


@pytest.mark.parametrize("render", [False, True])
def test_deltas_sum_to_box_length_and_samples_stay_in_their_tile(render):
    w = W.get("tiny_window")
    cams = W.cameras(w)
    pix = W.batch(w, cams, 4)
    win = w.window()
    o, d = camera.rays(cams, pix, win.origin, 0.0, w.tile[2])
    wf = sampler.window_f32(win)
    seg = sampler.segments(o, d, wf, w.K_ray, w.K_min, w.K_max)
    smp = sampler.stratified(o, d, seg, wf, seed=0, iteration=3, render=render)
    assert len(smp.t) == seg.ray_off[-1]
    for i in np.flatnonzero(seg.ray_ok):
        a, b = seg.ray_off[i], seg.ray_off[i + 1]
        sdt = smp.dt[a:b].astype(np.float64).sum()
        L = float(seg.t_out[i]) - float(seg.t_in[i])
        assert abs(sdt - L) <= 1e-5 * L
        assert np.all(np.diff(smp.t[a:b]) >= 0)
        assert smp.t[a] >= seg.t_in[i] and smp.t[b - 1] <= seg.t_out[i]
    assert np.all((smp.xyz >= 0) & (smp.xyz <= 1))
    # the FP64 point of each sample lies in the tile its slot names
    p = o[smp.ray].astype(np.float64) + smp.t.astype(np.float64)[:, None] * d[smp.ray].astype(np.float64)
    ix = np.floor(p[:, 0] / w.tile[0]).clip(0, 1)
    iy = np.floor(p[:, 1] / w.tile[1]).clip(0, 1)
    tile = (iy * 2 + ix).astype(int)
    frac_x = p[:, 0] / w.tile[0] - np.round(p[:, 0] / w.tile[0])
    frac_y = p[:, 1] / w.tile[1] - np.round(p[:, 1] / w.tile[1])
    clear = (np.abs(frac_x) > 1e-5) & (np.abs(frac_y) > 1e-5)
    assert np.all(tile[clear] == smp.slot[clear])
    if render:
        # bin centres: t = t0 + (k + 1/2) w
        i = np.flatnonzero(seg.ray_ok)[0]
        a = seg.ray_off[i]
        k = int(seg.K[i, 0])
        wbin = (float(seg.t1[i, 0]) - float(seg.t0[i, 0])) / k
        assert np.allclose(smp.t[a:a + k], float(seg.t0[i, 0]) + (np.arange(k) + 0.5) * wbin, rtol=1e-5)
