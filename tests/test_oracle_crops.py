"""Pins of the oracle's crops, ray pool and batch draw (oracle/crops.py), CPU
only: projections invert the localisation, the affine case is a closed-form
linear solve, every corner lies in its crop, the pool is exactly the accepted
pixels of the crops (brute force over the rectangles), and draws are the
Philox words' index formula, uniform over the pool."""
import numpy as np
import pytest

import synth
from synth import workloads as W
from oracle import camera, crops as C, philox, sampler


@pytest.mark.parametrize("name", ["tiny_sweep", "window2x2_full", "tile256_fp32"])
def test_projection_inverts_the_localisation(name):
    w = W.get(name)
    rng = np.random.default_rng(1)
    lo, hi = w.scene_box()
    for cam in W.cameras(w)[:6]:
        x = rng.uniform(lo[0], hi[0], 50)
        y = rng.uniform(lo[1], hi[1], 50)
        h = rng.uniform(lo[2], hi[2], 50)
        row, col = C.project(cam, x, y, h)
        xx, yy = camera.localise(cam, row, col, h)
        assert np.max(np.abs(xx - x)) < 1e-8 and np.max(np.abs(yy - y)) < 1e-8


def test_rpc_without_perturbation_projects_like_its_affine_part():
    w = W.get("tiny_sweep")
    for cam in W.cameras(w)[:3]:
        aff = synth.Camera(synth.CAM_AFFINE, cam.width, cam.height, a=cam.a.copy(), b=cam.b.copy())
        rpc = synth.rpc_as_affine(aff)
        x, y, h = np.array([3.0, 50.0]), np.array([7.0, 20.0]), np.array([2.0, 20.0])
        ra, ca = C.project(aff, x, y, h)
        rr, cr = C.project(rpc, x, y, h)
        assert np.allclose(ra, rr, atol=1e-7) and np.allclose(ca, cr, atol=1e-7)


def test_every_corner_lies_in_its_crop_and_the_view_crop_bounds_the_tiles():
    w = W.get("tiny_sweep")
    cams = W.cameras(w)
    for pos in [(0, 0), (1, 1)]:
        win = w.window(pos)
        tiles, views, proj = C.crops(cams, win, 2)
        for cam, rects, vr, pr in zip(cams, tiles, views, proj):
            for (r0, c0, h, wd), p in zip(rects, pr):
                inside = (p[:, 0] >= 0) & (p[:, 0] < cam.height) & (p[:, 1] >= 0) & (p[:, 1] < cam.width)
                assert np.all(p[inside, 0] >= r0) and np.all(p[inside, 0] <= r0 + h)
                assert np.all(p[inside, 1] >= c0) and np.all(p[inside, 1] <= c0 + wd)
                if h > 0 and wd > 0:
                    assert vr[0] <= r0 and vr[1] <= c0 and r0 + h <= vr[0] + vr[2] and c0 + wd <= vr[1] + vr[3]


def test_pool_is_the_accepted_pixels_of_the_crops():
    w = W.get("tiny_sweep")
    cams = W.cameras(w)
    win = w.window((1, 0))
    _, views, _ = C.crops(cams, win, 2)
    pool = C.ray_pool(cams, win, views)
    assert np.all(np.diff(pool.astype(np.int64)) > 0)  # strictly increasing: (view, row, col) order
    wf = sampler.window_f32(win)
    # brute force: every pixel of every crop, one at a time, through the sampler's segments
    want = []
    for v, (r0, c0, h, wd) in enumerate(views):
        for r in range(r0, r0 + h, 7):
            for c in range(c0, c0 + wd, 7):
                p = synth.pack_pixel(np.array([v]), np.array([r]), np.array([c]))
                o, d = camera.rays(cams, p, win.origin, win.origin[2], win.origin[2] + win.tile_size[2])
                if sampler.segments(o, d, wf, 4, 1, 4).ray_ok[0]:
                    want.append(int(p[0]))
    sub = set(int(x) for x in pool)
    stride = {int(x) for x in pool if ((int(x) >> 12) & 0xFFF) % 7 == views[int(x) >> 24][0] % 7
              and (int(x) & 0xFFF) % 7 == views[int(x) >> 24][1] % 7}
    assert set(want) == stride and set(want) <= sub and len(want) > 10


def test_draw_follows_the_index_formula_and_is_uniform():
    pool = np.arange(1000, dtype=np.uint32) * 3
    d = C.draw(pool, 40000, 9, 4)
    words = philox.philox4x32(np.array([[0, 0, 0, 0]], np.uint32), np.array([9, 4], np.uint32))[0]
    assert d[0] == pool[(int(words[0]) >> 8) * 1000 >> 24] and d[3] == pool[(int(words[3]) >> 8) * 1000 >> 24]
    counts = np.bincount((d // 3).astype(np.int64), minlength=1000)
    chi2 = ((counts - 40.0) ** 2 / 40.0).sum()
    assert chi2 < 1200  # 999 degrees of freedom
    assert np.array_equal(d, C.draw(pool, 40000, 9, 4)) and not np.array_equal(d, C.draw(pool, 40000, 9, 5))
