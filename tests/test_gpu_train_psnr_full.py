"""Equal quality at the model the speed-up is quoted on: the binary32 per-tile path and the
mixed-precision batched path, trained from the same initial weights on the same ray batches,
reach the same held-out PSNR on the 2x2 window of four 512 m tiles, each with its own L16,
T 2^19, 16 -> 2048 hash grid (FP16 working copy on the mixed path) and density MLP, and the
shared colour MLP.

Scene and views are the benchmark window's (sinusoid heightfield, 16 RPC views of 2048 px).
Views 1..15 train: a pool of 786,432 pixels drawn uniformly over their images, targets rendered
by the FP64 oracle at those pixels; every step draws 32,768 rays from the pool (the same
batches for both paths).  View 0 is held out: a 256 x 256 grid of its pixels (every 8th row and
column), rendered at bin centres; PSNR over the pixels whose rays the window accepts.

Per path, SEEDS jitter seeds of STEPS steps; the difference of the mean held-out PSNRs must be
within 0.1 dB (the benchmark metric's condition), its standard error printed beside it.  Both
paths follow the same learning-rate schedule: I-NGP's constant 1e-2, then over the last
DECAY_STEPS steps a cosine decay to 1e-4.  At a constant rate the last iterate wanders: held-out
PSNRs of runs that differ only in the jitter seed spread over 0.3-0.7 dB (measured: 37.0-38.7 dB
over four seeds), which no affordable number of seeds averages down to a 0.1 dB comparison; the
decay lets every run settle."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import step as OS, targets as OT
import synth
from synth import unpack_pixel, workloads as W
from gpu_util import model_config

pytestmark = pytest.mark.gpu
STEPS = 800
DECAY_STEPS = 300
RAYS = 32768
POOL = 786432
SEEDS = [41, 42, 43, 44, 45]


def lr_at(i, steps=STEPS, decay=DECAY_STEPS, lr0=1e-2, lr1=1e-4):
    """Learning rate of step i: lr0, then a cosine from lr0 to lr1 over the last `decay` steps."""
    k = i - (steps - decay)
    if decay <= 0 or k < 0:
        return lr0
    return lr1 + 0.5 * (lr0 - lr1) * (1.0 + np.cos(np.pi * (k + 1) / decay))


def equal_psnr_study(steps=STEPS, seeds=SEEDS, decay=DECAY_STEPS):
    """Held-out PSNR of the untrained model and, per path, of each seed's trained model."""
    build.build()
    assert torch.cuda.is_available()
    w = dataclasses.replace(W.get("window2x2_full"), n_rays=RAYS)
    cams = W.cameras(w)
    hf = W.scene(w)
    cfg = model_config(w)
    lay = cfg.grid()
    params = W.init_params(lay.n_params, cfg.geo_shapes(), cfg.col_shapes(), cfg.n_slots, cfg.n_colour_blocks(), 3)
    # training pool over views 1..15 and its targets (oracle), written into full-image crops
    pool = synth.random_pixels(2024, POOL, cams, views=np.arange(1, len(cams)))
    top, d = OT.rays_fp64(cams, pool, np.zeros(3), hf.lo[2], hf.hi[2])
    col = OT.shade_rays(hf, top, d).astype(np.float32)
    v, r, c = unpack_pixel(pool)
    crops = []
    for vi, cam in enumerate(cams):
        img = np.zeros((cam.crop[2], cam.crop[3], 3), np.float32)
        m = v == vi
        img[r[m] - cam.crop[0], c[m] - cam.crop[1]] = col[m]
        crops.append(torch.from_numpy(img).cuda())
    rng = np.random.default_rng(7)
    batches = torch.from_numpy(pool[rng.integers(0, POOL, (steps, RAYS))].view(np.int32)).cuda()
    # held-out view 0
    c0 = cams[0]
    rr, cc = np.meshgrid(np.arange(4, c0.height, 8), np.arange(4, c0.width, 8), indexing="ij")
    held = synth.pack_pixel(np.zeros(rr.size, int), rr.ravel(), cc.ravel())
    _, _, seg, _ = OS.sample_rays(cfg, cams, w.window(), held, 0, 0, True)
    ok = seg.ray_ok.astype(bool)
    ht, hd = OT.rays_fp64(cams, held, np.zeros(3), hf.lo[2], hf.hi[2])
    gt = OT.shade_rays(hf, ht, hd)[ok]
    held_t = torch.from_numpy(held.view(np.int32)).cuda()
    ctx = snk.Context(0)
    ctx.set_views(cams, crops)
    win = snk.window_struct(w.window())
    sp0 = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 0, 0)
    ctx.reserve(max(RAYS, len(held)), ctx.max_samples(win, sp0, max(RAYS, len(held))))

    def held_out_psnr(tr):
        tr.sampler = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 1, 0, 0)
        out = torch.zeros(len(held) * 5, dtype=torch.float32, device="cuda")
        tr.render(held_t, out)
        rgb = out.cpu().numpy().reshape(-1, 5)[ok, :3].astype(np.float64)
        return float(-10.0 * np.log10(np.mean((rgb - gt) ** 2)))

    psnr0 = held_out_psnr(Trainer(ctx, model_from_workload(w, snk.SNK_FP32), win, sp0, params))
    psnr = {}
    for name, prec in (("fp32", snk.SNK_FP32), ("mixed", snk.SNK_MIXED)):
        model = model_from_workload(w, prec)
        vals = []
        for seed in seeds:
            tr = Trainer(ctx, model, win, snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, seed, 0), params)
            for i in range(steps):
                tr.adam = snk.adam_struct(lr=lr_at(i, steps, decay))
                tr.train_step(batches[i])
            assert ctx.sync_status(tr.state) == snk.SNK_OK
            vals.append(held_out_psnr(tr))
            del tr
        psnr[name] = np.array(vals)
    ctx.close()
    return psnr0, psnr


def test_fp32_per_tile_and_mixed_batched_reach_equal_psnr_at_full_model_size():
    psnr0, psnr = equal_psnr_study()
    d = psnr["mixed"] - psnr["fp32"]
    delta = float(d.mean())
    se = float(d.std(ddof=1) / np.sqrt(len(d)))
    print("held-out PSNR at the 2x2 window's full model (untrained %.2f dB), %d seeds x %d steps of %d rays: "
          "fp32 %s, mixed %s, difference %.3f dB (SE %.3f dB)" % (psnr0, len(SEEDS), STEPS, RAYS,
                                                                 np.round(psnr["fp32"], 3), np.round(psnr["mixed"], 3),
                                                                 delta, se))
    assert psnr["fp32"].mean() > psnr0 + 6.0, "training did not reach a usable fit"
    assert abs(delta) <= 0.1, (delta, se)
