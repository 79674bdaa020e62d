"""Occupancy culling (Sec. 4.1, SAT-NGP's coarse voxel grid) on the device
against the oracle: culled sampling bit-exact for a given grid, a training
step with culling within the binary32 tolerances, the grid update's densities
within the path's tolerance and its occupied flags equal except within rounding
of the threshold; and training with periodic updates culls empty space."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import occupancy as O, step as OS
from gpu_util import GRAD_REL_FP32, RGB_REL_FP32, RGB_REL_MIXED, close, gpu_to_ray_major, make_case, normwise

pytestmark = pytest.mark.gpu
R = 16


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _grid(n_slots, seed, frac=0.55):
    """Blocky random grid: 4^3-cell blocks occupied with probability frac."""
    rng = np.random.default_rng(seed)
    blk = rng.random((n_slots, R // 4, R // 4, R // 4)) < frac
    g = blk.repeat(4, 1).repeat(4, 2).repeat(4, 3)        # (slot, z, y, x)
    return g.reshape(n_slots, -1)


@pytest.mark.parametrize("name,n_rays", [("tiny_window", 160), ("window2x2_full", 700), ("tile512_full", 300)])
def test_culled_sampling_is_bit_exact(ctx, name, n_rays):
    case = make_case(name, n_rays=n_rays, with_targets=False)
    w = case.w
    ctx.set_views(case.cams)
    occ = _grid(w.n_slots, 4)
    occ_t = dev(occ.astype(np.uint8))
    B = n_rays
    nseg = 1 + (w.nx == 2) + (w.ny == 2)
    cap = B * nseg * w.K_max + 512
    f32, i32, u8 = torch.float32, torch.int32, torch.uint8
    g = {k: torch.zeros(n, dtype=t, device="cuda") for k, n, t in
         [("ray_od", 6 * B, f32), ("ray_ok", B, u8), ("seg_slot", 3 * B, u8), ("seg_t", 6 * B, f32),
          ("seg_n", 3 * B, i32), ("seg_off", 3 * B, i32), ("smp_t", cap, f32), ("smp_dt", cap, f32),
          ("smp_xyz", 3 * cap, f32), ("state", snk.STATE_WORDS, i32)]}
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 7, 3, occupancy=occ_t, occ_res=R)
    ctx.call("snk_sample_segments", ctypes.byref(snk.window_struct(w.window())), snk.ptr(dev(case.pix.view(np.int32))),
             B, ctypes.byref(sp), *[snk.ptr(g[k]) for k in ("ray_od", "ray_ok", "seg_slot", "seg_t", "seg_n",
                                                            "seg_off", "smp_t", "smp_dt", "smp_xyz")],
             cap, snk.ptr(g["state"]), None)
    torch.cuda.synchronize()
    h = {k: v.cpu().numpy() for k, v in g.items()}
    _, _, seg, smp = OS.sample_rays(case.cfg, case.cams, w.window(), case.pix, 7, 3, False, occ=(occ, R))
    _, _, seg_all, _ = OS.sample_rays(case.cfg, case.cams, w.window(), case.pix, 7, 3, False)
    assert 0 < seg.ray_off[-1] < seg_all.ray_off[-1]  # the grid removes some samples, not all
    seg_n = h["seg_n"].reshape(B, 3)
    assert np.array_equal(seg_n, seg.K)
    assert int(h["state"][3:4].view(np.uint32)[0]) == int(seg.ray_off[-1])
    idx = gpu_to_ray_major(seg_n, h["seg_off"].reshape(B, 3), seg.ray_off)
    assert np.array_equal(h["smp_t"][idx], smp.t) and np.array_equal(h["smp_dt"][idx], smp.dt)
    assert np.array_equal(h["smp_xyz"].reshape(-1, 3)[idx], smp.xyz)


def test_train_step_with_culling_matches_oracle(ctx):
    case = make_case("tiny_window", n_rays=160, table_scale=0.3)
    w = case.w
    crops = [dev(t.astype(np.float32)) for t in case.targets]
    ctx.set_views(case.cams, crops)
    occ = _grid(w.n_slots, 9)
    occ_t = dev(occ.astype(np.uint8))  # the sampler holds a raw pointer: keep the tensor alive
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 5, 0, occupancy=occ_t, occ_res=R)
    tr = Trainer(ctx, model_from_workload(w, snk.SNK_FP32), snk.window_struct(w.window()), sp, case.params)
    out = torch.zeros(160 * 5, dtype=torch.float32, device="cuda")
    tr.train_step(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    n = len(case.params)
    ref = OS.train_step(case.cfg, case.params.astype(np.float64), np.zeros(n), np.zeros(n),
                        [0] * case.cfg.n_optimisers(), case.cams, w.window(), case.pix, case.targets, 5, 0,
                        occ=(occ, R))
    st = tr.read_state()
    assert st["n_samples"] == int(ref.seg.ray_off[-1])
    go = out.cpu().numpy().reshape(160, 5)
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        good, err = close(a, b, RGB_REL_FP32)
        assert good, (nm, err)
    m = tr.m.cpu().numpy().astype(np.float64)
    for a, b, mlp_a in OS.group_ranges(case.cfg):
        assert normwise(m[a:b], ref.m[a:b]) < GRAD_REL_FP32


@pytest.mark.parametrize("precision", [snk.SNK_FP32, snk.SNK_MIXED])
def test_occupancy_update_matches_oracle(ctx, precision):
    case = make_case("tiny_window", n_rays=16, table_scale=0.5, with_targets=False)
    w = case.w
    model = model_from_workload(w, precision)
    tr = Trainer(ctx, model, snk.window_struct(w.window()), snk.sampler_struct(8, 8, 8), case.params)
    n = R ** 3
    dens = torch.zeros(w.n_slots * n, dtype=torch.float32, device="cuda")
    occ = torch.ones(w.n_slots * n, dtype=torch.uint8, device="cuda")
    wc = case.params.astype(np.float64)
    tol = 1e-5
    if precision == snk.SNK_MIXED:
        wc = case.params.astype(np.float16).astype(np.float64)
        tol = RGB_REL_MIXED
    ref = np.zeros((w.n_slots, n))
    for step, (seed, decay, thr) in enumerate([(3, 0.95, 0.01), (4, 0.5, 50.0)]):
        ctx.call("snk_occupancy_update", ctypes.byref(model), ctypes.byref(tr.p_struct), snk.ptr(dens), snk.ptr(occ),
                 R, decay, thr, seed, step, None)
        torch.cuda.synchronize()
        ref, ref_occ = O.update(case.cfg, wc, ref, R, decay, thr, seed, step)
        gd = dens.cpu().numpy().reshape(w.n_slots, n).astype(np.float64)
        assert np.all(np.abs(gd - ref) <= tol * np.maximum(np.abs(ref), 1e-3)), (step, np.max(np.abs(gd - ref) / ref))
        go = occ.cpu().numpy().reshape(w.n_slots, n).astype(bool)
        for k in range(w.n_slots):
            t = min(thr, ref[k].mean())
            sure = np.abs(ref[k] - t) > 4 * tol * t
            assert np.array_equal(go[k][sure], ref_occ[k][sure]), (step, k)
        if step == 1:
            assert 0 < go.mean() < 1  # the second threshold splits the grid


def test_training_with_updates_culls_empty_space(ctx):
    """Train on fresh random batches with a grid update every 25 steps; the samples
    of a fixed batch rendered through the grid drop as the field learns empty air.
    Decay 0.5: in a 600-step run a slower decay keeps the densities of the first
    update (taken near the initial sigma = exp(0) = 1) above the threshold."""
    import synth
    case = make_case("tiny_window", n_rays=160, table_scale=1e-4)
    w = case.w
    crops = [dev(t.astype(np.float32)) for t in case.targets]
    ctx.set_views(case.cams, crops)
    n = R ** 3
    dens = torch.zeros(w.n_slots * n, dtype=torch.float32, device="cuda")
    occ = torch.ones(w.n_slots * n, dtype=torch.uint8, device="cuda")
    model = model_from_workload(w, snk.SNK_MIXED)
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 5, 0, occupancy=occ, occ_res=R)
    tr = Trainer(ctx, model, snk.window_struct(w.window()), sp, case.params)
    eval_pix = dev(case.pix.view(np.int32))
    out = torch.zeros(len(case.pix) * 5, dtype=torch.float32, device="cuda")

    def rendered_samples():
        tr.render(eval_pix, out)
        return tr.read_state()["n_samples"]

    n0 = rendered_samples()
    for i in range(600):
        tr.train_step(dev(synth.random_pixels(1000 + i, 1024, case.cams).view(np.int32)))
        if i >= 100 and i % 25 == 0:
            ctx.call("snk_occupancy_update", ctypes.byref(model), ctypes.byref(tr.p_struct), snk.ptr(dens),
                     snk.ptr(occ), R, 0.5, 0.01, 11, i, None)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    n1 = rendered_samples()
    frac = occ.float().mean().item()
    print("rendered samples of the fixed batch: %d -> %d; occupied cells %.3f" % (n0, n1, frac))
    assert frac < 0.9 and n1 < 0.9 * n0
    assert np.isfinite(tr.read_state()["loss"])
