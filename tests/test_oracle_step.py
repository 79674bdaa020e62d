"""Pins of the oracle's whole training step: the analytic gradient of the full
pipeline (rays -> segments -> encoding -> MLPs -> rendering -> loss) against
FP64 central differences, the Adam bookkeeping per optimiser, and the target
renderer against a closed form (CPU only)."""
import numpy as np
import pytest

import synth
from synth import workloads as W
from oracle import step as OS, targets as OT, camera, render, hashgrid


def model_config(w):
    return OS.ModelConfig(L=w.L, F=w.F, log2_T=w.log2_T, n_min=w.n_min, n_max=w.n_max, hidden=w.hidden,
                          geo_out=w.geo_out, colour=w.colour, shared_colour=w.shared_colour, n_slots=w.n_slots,
                          K_ray=w.K_ray, K_min=w.K_min, K_max=w.K_max)


def _setup(name, n_rays, hidden=16, seed=0):
    w = W.get(name, n_rays=n_rays, hidden=hidden)
    cams = W.cameras(w)
    tg = OT.render_targets(W.scene(w), cams)
    cfg = model_config(w)
    lay = cfg.grid()
    flat = W.init_params(lay.n_params, cfg.geo_shapes(), cfg.col_shapes(), cfg.n_slots, cfg.n_colour_blocks(),
                         seed).astype(np.float64)
    # larger table values than the NGP init so that the features matter
    rng = np.random.default_rng(seed)
    for a, b, mlp_a in OS.group_ranges(cfg)[:cfg.n_slots]:
        flat[a:mlp_a] = rng.uniform(-0.5, 0.5, mlp_a - a)
    pix = W.batch(w, cams, seed + 11)
    return w, cams, tg, cfg, flat, pix


def _loss(cfg, flat, cams, win, pix, tg, seed, it):
    o, d, seg, smp = OS.sample_rays(cfg, cams, win, pix, seed, it, False)
    sigma, rgb_s, _ = OS.field_forward(cfg, flat, smp)
    rgb, _, _, _, _ = render.composite(sigma, rgb_s, smp.t.astype(np.float64), smp.dt.astype(np.float64),
                                       seg.ray_off)
    gt = OS.gather_targets(cams, pix, tg)
    return render.mse_loss(rgb, gt, seg.ray_ok)[0]


@pytest.mark.parametrize("name", ["tiny_tile", "tiny_window"])
def test_full_step_gradient_matches_central_differences(name):
    w, cams, tg, cfg, flat, pix = _setup(name, 24)
    n = len(flat)
    res = OS.train_step(cfg, flat, np.zeros(n), np.zeros(n), [0] * cfg.n_optimisers(), cams, w.window(), pix,
                        tg, 5, 9)
    rng = np.random.default_rng(0)
    lay = cfg.grid()
    picks = []
    for a, b, mlp_a in OS.group_ranges(cfg):
        g_abs = np.abs(res.grad[a:mlp_a]) if mlp_a > a else np.zeros(0)
        if g_abs.size:                                   # table entries that receive gradient
            nz = np.flatnonzero(g_abs > 1e-9)
            picks += list(a + rng.choice(nz, min(6, nz.size), replace=False))
        picks += list(rng.integers(mlp_a, b, 6))         # MLP weights
    for p in picks:
        h = 1e-6 * max(1.0, abs(flat[p]))
        fp_ = flat.copy()
        fp_[p] += h
        fm_ = flat.copy()
        fm_[p] -= h
        fd = (_loss(cfg, fp_, cams, w.window(), pix, tg, 5, 9) - _loss(cfg, fm_, cams, w.window(), pix, tg, 5, 9)) / (2 * h)
        assert abs(fd - res.grad[p]) <= 1e-6 * abs(fd) + 1e-10, (p, fd, res.grad[p])


def test_step_updates_every_optimiser_and_counts_steps():
    w, cams, tg, cfg, flat, pix = _setup("tiny_window", 40)
    n = len(flat)
    steps = [3] * cfg.n_optimisers()
    res = OS.train_step(cfg, flat, np.zeros(n), np.zeros(n), steps, cams, w.window(), pix, tg, 1, 2)
    assert res.extra["steps"] == [4] * cfg.n_optimisers()
    assert cfg.n_optimisers() == 5                       # 4 tiles + 1 shared colour net
    moved = res.params != flat
    assert np.array_equal(moved, res.grad + 0 != 0) or np.all(moved[res.grad != 0])
    # a parameter with zero gradient and zero moments does not move (no decay on tables)
    lay = cfg.grid()
    a, b, mlp_a = OS.group_ranges(cfg)[0]
    z = np.flatnonzero(res.grad[a:mlp_a] == 0)
    assert z.size > 0 and np.all(res.params[a + z] == flat[a + z])


def test_target_renderer_flat_ground_closed_form():
    """Flat ground z = z_base: the hit lies at t = (z_max - z_base) / cos(theta)
    and the colour is albedo * (0.2 + 0.8 s_z)."""
    lo, hi = np.zeros(3), np.array([100.0, 100.0, 40.0])
    hf = synth.heightfield(0, lo, hi)
    hf.amp = np.zeros_like(hf.amp)
    cams = synth.pushbroom_cameras(2, 2, 32, 32, lo, hi)
    pix = synth.pack_pixel([0, 1, 1], [10, 16, 20], [12, 16, 5])
    o, d = camera.rays_fp64(cams, pix, np.zeros(3), 0.0, 40.0)
    col = OT.shade_rays(hf, o, d)
    t_hit = (40.0 - hf.z_base) / (-d[:, 2])
    p = o + t_hit[:, None] * d
    inside = np.all((p[:, :2] >= 0) & (p[:, :2] <= 100), axis=1)
    expect = OT.albedo(hf, p[:, 0], p[:, 1]) * (0.2 + 0.8 * hf.sun[2])
    assert inside.any()
    assert np.allclose(col[inside], expect[inside], atol=1e-7)
    # the hit distance itself (the depth a perfect model renders), NaN outside the box
    t = OT.surface_t(hf, o, d)
    assert np.allclose(t[inside], t_hit[inside], rtol=0, atol=1e-8)
    assert np.all(np.isnan(t[~inside]))
