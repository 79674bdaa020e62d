"""Pins of the oracle's occupancy grid and culling (oracle/occupancy.py), CPU
only: update points lie in their own cells, culling with a full grid changes
nothing and with an empty grid leaves no samples, a culled sample renders
exactly like a sample of zero density, and the update rule on a constant field
gives closed-form densities and thresholds."""
import dataclasses

import numpy as np
import pytest

from synth import workloads as W
from oracle import occupancy as O, render, step as OS

R = 8


def _case(n_rays=48):
    w = W.get("tiny_window", n_rays=n_rays)
    cams = W.cameras(w)
    cfg = OS.ModelConfig(L=w.L, F=w.F, log2_T=w.log2_T, n_min=w.n_min, n_max=w.n_max, hidden=16,
                         geo_out=w.geo_out, colour=w.colour, shared_colour=w.shared_colour, n_slots=w.n_slots,
                         K_ray=w.K_ray, K_min=w.K_min, K_max=w.K_max)
    lay = cfg.grid()
    flat = W.init_params(lay.n_params, cfg.geo_shapes(), cfg.col_shapes(), cfg.n_slots, cfg.n_colour_blocks(),
                         0).astype(np.float64)
    rng = np.random.default_rng(0)
    for a, b, mlp_a in OS.group_ranges(cfg)[:cfg.n_slots]:
        flat[a:mlp_a] = rng.uniform(-0.5, 0.5, mlp_a - a)
    return w, cams, cfg, flat, W.batch(w, cams, 3)


def test_update_points_lie_in_their_cells():
    for k in range(3):
        p = O.points(k, R, 5, 7)
        assert np.array_equal(O.cells(p, R), np.arange(R ** 3))
    assert not np.array_equal(O.points(0, R, 5, 7), O.points(0, R, 5, 8))


def test_full_grid_changes_nothing_and_empty_grid_leaves_nothing():
    w, cams, cfg, flat, pix = _case()
    o, d, seg, smp = OS.sample_rays(cfg, cams, w.window(), pix, 1, 0, False)
    full = np.ones((cfg.n_slots, R ** 3), bool)
    _, _, seg_f, smp_f = OS.sample_rays(cfg, cams, w.window(), pix, 1, 0, False, occ=(full, R))
    assert np.array_equal(seg_f.K, seg.K) and np.array_equal(seg_f.ray_off, seg.ray_off)
    assert np.array_equal(smp_f.t, smp.t) and np.array_equal(smp_f.xyz, smp.xyz)
    _, _, seg_e, smp_e = OS.sample_rays(cfg, cams, w.window(), pix, 1, 0, False, occ=(~full, R))
    assert len(smp_e.t) == 0 and np.all(seg_e.ray_off == 0) and np.all(seg_e.K == 0)


def test_a_culled_sample_renders_like_a_sample_of_zero_density():
    w, cams, cfg, flat, pix = _case()
    occ = np.random.default_rng(2).random((cfg.n_slots, R ** 3)) < 0.6
    o, d, seg, smp = OS.sample_rays(cfg, cams, w.window(), pix, 1, 0, False)
    keep = occ[smp.slot, O.cells(smp.xyz, R)]
    sigma, rgb_s, _ = OS.field_forward(cfg, flat, smp)
    zeroed = np.where(keep, sigma, 0.0)
    want = render.composite(zeroed, rgb_s, smp.t.astype(np.float64), smp.dt.astype(np.float64), seg.ray_off)
    seg_c, smp_c = O.cull(seg, smp, occ, R)
    assert 0 < len(smp_c.t) < len(smp.t)
    sigma_c, rgb_c, _ = OS.field_forward(cfg, flat, smp_c)
    got = render.composite(sigma_c, rgb_c, smp_c.t.astype(np.float64), smp_c.dt.astype(np.float64), seg_c.ray_off)
    for a, b in zip(got[:3], want[:3]):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def test_update_rule_on_a_constant_field():
    w, cams, cfg, flat, _ = _case()
    # density output row of W3 set to zero: g0 = 0, sigma = exp(0) = 1 at every point
    tiles, _ = OS.unflatten(cfg, flat)
    for k in range(cfg.n_slots):
        tiles[k][1][2][0, :] = 0.0
    n = R ** 3
    dens, occ = O.update(cfg, flat, np.zeros((cfg.n_slots, n)), R, 0.95, 0.01, 1, 0)
    assert np.allclose(dens, 1.0, rtol=0, atol=1e-15) and occ.all()
    # half the cells start at 10: they decay to 9.5, the rest rise to 1; mean 5.25
    d0 = np.zeros((cfg.n_slots, n))
    d0[:, ::2] = 10.0
    dens, occ = O.update(cfg, flat, d0, R, 0.95, 2.0, 1, 1)
    assert np.allclose(dens[:, ::2], 9.5) and np.allclose(dens[:, 1::2], 1.0)
    assert occ[:, ::2].all() and not occ[:, 1::2].any()          # threshold min(2, 5.25) = 2
    dens, occ = O.update(cfg, flat, d0, R, 0.95, 100.0, 1, 1)
    assert occ[:, ::2].all() and not occ[:, 1::2].any()          # threshold min(100, 5.25) = 5.25
    dens, occ = O.update(cfg, flat, d0, R, 0.95, 0.5, 1, 1)
    assert occ.all()                                              # threshold 0.5: every cell above
