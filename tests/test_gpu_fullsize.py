"""The headline step at full size, in the launch configuration bench.py times
(2x2 window, 524,288 rays, ~64 M samples, mixed path, autotuned shapes),
checked where the oracle can follow it one item at a time and by properties
that hold at any size:

* sampling: the full batch's segments and samples of a random subset of rays
  bit-exact against the oracle's sampler (same batch indices, same jitter);
* rendering: the step's rendered colour, depth and opacity of a random subset
  of rays against the oracle's forward on the FP16 working copy, with the
  training jitter of those rays (mixed-path tolerance);
* the first Adam step: every parameter whose gradient is far above eps moves by
  lr against its sign (m_hat / sqrt(v_hat) = +-1), none moves by more, and one
  with a zero gradient stays;
* the backward reading the stored activations and the one recomputing them
  compute the same step."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import step as OS
from synth import workloads as W
from gpu_util import RGB_REL_MIXED, close, model_config, normwise

pytestmark = pytest.mark.gpu
N_CHECK = 48  # rays the oracle follows


@pytest.fixture(scope="module")
def setup():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    ctx = snk.Context(0)
    w = W.get("window2x2_full")
    model = model_from_workload(w)
    lay = snk.layout(model)
    cams, targets, params = bench.make_inputs(w, lay.grid_params)
    cfg = model_config(w)
    # a non-trivial field: random tables (the bench's are near zero)
    rng = np.random.default_rng(7)
    for a, b, mlp_a in OS.group_ranges(cfg)[:cfg.n_slots]:
        params[a:mlp_a] = rng.uniform(-0.3, 0.3, mlp_a - a).astype(np.float32)
    crops = [torch.from_numpy(t).cuda() for t in targets]
    ctx.set_views(cams, crops)
    pix = W.batch(w, cams, 50)
    pix_t = torch.from_numpy(pix.view(np.int32)).cuda()
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 1234, 0)
    win = snk.window_struct(w.window())
    ctx.reserve(w.n_rays, ctx.max_samples(win, sp, w.n_rays))
    tr = Trainer(ctx, model, win, sp, params)
    tuning = tr.autotune(pix_t)
    yield dict(ctx=ctx, w=w, model=model, cams=cams, params=params, cfg=cfg, pix=pix, pix_t=pix_t, sp=sp, win=win,
               tuning=tuning, crops=crops)
    ctx.close()


def test_full_batch_sampling_is_bit_exact_on_sampled_rays(setup):
    ctx, w, pix = setup["ctx"], setup["w"], setup["pix"]
    B = len(pix)
    cap = ctx.max_samples(setup["win"], setup["sp"], B)
    f32, i32, u8 = torch.float32, torch.int32, torch.uint8
    g = {k: torch.zeros(n, dtype=t, device="cuda") for k, n, t in
         [("ray_od", 6 * B, f32), ("ray_ok", B, u8), ("seg_slot", 3 * B, u8), ("seg_t", 6 * B, f32),
          ("seg_n", 3 * B, i32), ("seg_off", 3 * B, i32), ("smp_t", cap, f32), ("smp_dt", cap, f32),
          ("smp_xyz", 3 * cap, f32), ("state", snk.STATE_WORDS, i32)]}
    ctx.call("snk_sample_segments", ctypes.byref(setup["win"]), snk.ptr(setup["pix_t"]), B, ctypes.byref(setup["sp"]),
             *[snk.ptr(g[k]) for k in ("ray_od", "ray_ok", "seg_slot", "seg_t", "seg_n", "seg_off", "smp_t", "smp_dt",
                                       "smp_xyz")], cap, snk.ptr(g["state"]), None)
    assert ctx.sync_status(g["state"]) == snk.SNK_OK
    n_samples = int(g["state"][3:4].cpu().numpy().view(np.uint32)[0])
    assert 50e6 < n_samples < 80e6
    ids = np.sort(np.random.default_rng(3).choice(B, N_CHECK, replace=False))
    _, _, seg, smp = OS.sample_rays(setup["cfg"], setup["cams"], w.window(), pix[ids], 1234, 0, False, ray_ids=ids)
    h = {k: g[k].cpu().numpy() for k in ("ray_ok", "seg_slot", "seg_t", "seg_n", "seg_off")}
    assert np.array_equal(h["ray_ok"][ids], seg.ray_ok)
    assert np.array_equal(h["seg_slot"].reshape(B, 3)[ids].astype(np.int64), seg.slot)
    seg_t = h["seg_t"].reshape(B, 3, 2)[ids]
    assert np.array_equal(seg_t[..., 0], seg.t0) and np.array_equal(seg_t[..., 1], seg.t1)
    seg_n = h["seg_n"].reshape(B, 3)[ids]
    assert np.array_equal(seg_n, seg.K)
    # the sampled rays' samples, gathered from the slot-major buffers in ray order
    off = h["seg_off"].reshape(B, 3)[ids]
    idx = np.concatenate([off[i, s] + np.arange(seg_n[i, s]) for i in range(N_CHECK) for s in range(3)
                          if seg_n[i, s] > 0]).astype(np.int64)
    assert len(idx) == int(seg.ray_off[-1])
    it = torch.from_numpy(idx).cuda()
    assert np.array_equal(g["smp_t"][it].cpu().numpy(), smp.t)
    assert np.array_equal(g["smp_dt"][it].cpu().numpy(), smp.dt)
    assert np.array_equal(g["smp_xyz"].view(-1, 3)[it].cpu().numpy(), smp.xyz)


def _step(setup, saved):
    ctx = setup["ctx"]
    ctx.set_tuning(tc_bwd_saved=saved)
    tr = Trainer(ctx, setup["model"], setup["win"], setup["sp"], setup["params"])
    B = len(setup["pix"])
    out = torch.zeros(B * 5, dtype=torch.float32, device="cuda")
    tr.train_step(setup["pix_t"], out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    return tr, out.cpu().numpy().reshape(B, 5)


def test_full_batch_step_renders_sampled_rays_like_the_oracle_and_takes_the_first_adam_step(setup):
    w = setup["w"]
    saved = setup["tuning"]["tc_bwd_saved"]
    tr, out = _step(setup, saved)
    st = tr.read_state()
    assert np.isfinite(st["loss"]) and st["n_accepted"] > 0.9 * len(setup["pix"])
    # rendering of sampled rays: the oracle on the FP16 working copy, the training jitter of those rays
    ids = np.sort(np.random.default_rng(4).choice(len(setup["pix"]), N_CHECK, replace=False))
    wc = setup["params"].astype(np.float16).astype(np.float64)
    ref = OS.render_rays(setup["cfg"], wc, setup["cams"], w.window(), setup["pix"][ids], seed=1234, iteration=0,
                         render_mode=False, ray_ids=ids)
    for nm, a, b in [("rgb", out[ids, :3], ref.rgb), ("depth", out[ids, 3], ref.depth),
                     ("opacity", out[ids, 4], ref.opacity)]:
        ok, err = close(a, b, RGB_REL_MIXED)
        assert ok, (nm, err)
    # the first Adam step (bias-corrected m / sqrt(v) = sign(g)): moved by lr against m, or not at all
    p0 = setup["params"].astype(np.float64)
    p1 = tr.params.cpu().numpy().astype(np.float64)
    m1 = tr.m.cpu().numpy().astype(np.float64)
    lr = tr.adam.lr
    # |g| = 10 |m| >> eps = 1e-15 (eps / |g| <= 1e-5 here), so the move is lr to FP32 rounding
    big = np.abs(m1) > 1e-11
    assert (m1 != 0).mean() > 0.05 and big.sum() > 100000
    assert np.all(np.abs((p1 - p0)[big] + lr * np.sign(m1[big])) <= 1e-6 + 1e-6 * np.abs(p0[big]))
    assert np.all(p1[m1 == 0] == p0[m1 == 0])
    assert np.all(np.abs(p1 - p0) <= lr * (1 + 1e-5) + 1e-6 * np.abs(p0))


def test_stored_and_recomputed_activations_agree_at_full_size(setup):
    tr1, out1 = _step(setup, 1)
    tr0, out0 = _step(setup, 0)
    setup["ctx"].set_tuning(tc_bwd_saved=setup["tuning"]["tc_bwd_saved"])
    assert np.array_equal(out1, out0)
    assert normwise(tr1.m.cpu().numpy().astype(np.float64), tr0.m.cpu().numpy().astype(np.float64)) < 1e-5


def test_binary32_per_tile_step_renders_sampled_rays_like_the_oracle(setup):
    """The comparison arm of the headline metric: the binary32 path, one launch chain per
    tile, on the same full batch; rendered sampled rays within the binary32 tolerance of the
    oracle on the binary32 parameters."""
    from gpu_util import RGB_REL_FP32
    w = setup["w"]
    tr = Trainer(setup["ctx"], model_from_workload(w, snk.SNK_FP32), setup["win"], setup["sp"], setup["params"])
    B = len(setup["pix"])
    out = torch.zeros(B * 5, dtype=torch.float32, device="cuda")
    tr.train_step(setup["pix_t"], out)
    assert setup["ctx"].sync_status(tr.state) == snk.SNK_OK
    out = out.cpu().numpy().reshape(B, 5)
    ids = np.sort(np.random.default_rng(5).choice(B, N_CHECK, replace=False))
    ref = OS.render_rays(setup["cfg"], setup["params"].astype(np.float64), setup["cams"], w.window(),
                         setup["pix"][ids], seed=1234, iteration=0, render_mode=False, ray_ids=ids)
    for nm, a, b in [("rgb", out[ids, :3], ref.rgb), ("depth", out[ids, 3], ref.depth),
                     ("opacity", out[ids, 4], ref.opacity)]:
        ok, err = close(a, b, RGB_REL_FP32)
        assert ok, (nm, err)
