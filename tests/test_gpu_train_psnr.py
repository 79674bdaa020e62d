"""Equal quality of the two step implementations: the binary32 per-tile path and
the mixed-precision batched path, trained from the same initial weights on the
same ray batches (same jitter), reach the same held-out PSNR within 0.1 dB.

Scene: the small 2x2 window (four 48 m tiles, shared colour net), targets
rendered by the FP64 oracle.  Views 1..5 train; view 0 is held out and rendered
at bin centres."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
import synth
from synth import workloads as W
from oracle import targets as OT
from gpu_util import model_config

pytestmark = pytest.mark.gpu
STEPS = 400
RAYS = 2048


def psnr(a, b):
    return float(-10.0 * np.log10(np.mean((a - b) ** 2)))


def test_fp32_per_tile_and_mixed_batched_reach_equal_psnr():
    build.build()
    assert torch.cuda.is_available()
    w = dataclasses.replace(W.get("tiny_window"), n_views=6, n_rays=RAYS)
    cams = W.cameras(w)
    targets = OT.render_targets(W.scene(w), cams)
    cfg = model_config(w)
    lay = cfg.grid()
    params = W.init_params(lay.n_params, cfg.geo_shapes(), cfg.col_shapes(), cfg.n_slots, cfg.n_colour_blocks(), 3)
    train_views = np.arange(1, 6)
    batches = [synth.random_pixels(1000 + i, RAYS, cams, views=train_views) for i in range(STEPS)]
    c0 = cams[0]
    rr, cc = np.meshgrid(np.arange(c0.crop[2]), np.arange(c0.crop[3]), indexing="ij")
    held = synth.pack_pixel(np.zeros(rr.size, int), rr.ravel() + c0.crop[0], cc.ravel() + c0.crop[1])
    gt = targets[0].reshape(-1, 3).astype(np.float64)

    results = {}
    for name, prec in (("fp32", snk.SNK_FP32), ("mixed", snk.SNK_MIXED)):
        ctx = snk.Context(0)
        crops = [torch.from_numpy(t).cuda() for t in targets]
        ctx.set_views(cams, crops)
        model = model_from_workload(w, prec)
        tr = Trainer(ctx, model, snk.window_struct(w.window()), snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 9, 0),
                     params)
        for b in batches:
            tr.train_step(torch.from_numpy(b.view(np.int32)).cuda())
        assert ctx.sync_status(tr.state) == snk.SNK_OK
        out = torch.zeros(len(held) * 5, dtype=torch.float32, device="cuda")
        tr.sampler = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 1, 0, 0)
        tr.render(torch.from_numpy(held.view(np.int32)).cuda(), out)
        assert ctx.sync_status(tr.state) == snk.SNK_OK
        rgb = out.cpu().numpy().reshape(-1, 5)[:, :3].astype(np.float64)
        results[name] = (psnr(rgb, gt), tr.read_state()["loss"])
        ctx.close()
    print("held-out PSNR (dB), final loss:", results)
    init_psnr = psnr(np.zeros_like(gt), gt)
    assert results["fp32"][0] > init_psnr + 3.0, "training did not improve the held-out view"
    assert abs(results["fp32"][0] - results["mixed"][0]) <= 0.1, results
