"""Gradients of the mixed-precision step at the full model sizes the benchmark runs -- one tile
(L16, T 2^19, 16 -> 2048, geometry + colour MLPs, 16 RPC views of 1024 px) and the 2x2 window
(four such tiles, shared colour net, 16 views of 2048 px) -- on 4096-ray batches drawn over the
whole images, against the FP64 oracle on the model's FP16 working copy:

* every parameter group's gradient (via Adam's first moment) within 5e-3 norm-wise, and the MLP
  weight gradients element by element within rel 5e-3 (floor 5e-3 x max), after the exact
  effect of at most MAX_FLIPS binary32-ambiguous ReLU decisions is accounted for;
* one tile: the GPU's gradient along directions in the table, the density MLP, the colour MLP
  and its output layer against FP64 central differences of the oracle's loss (the batch's
  samples held fixed), within 5e-3, and the oracle's analytic gradient against the same
  differences (its own pin at full size): within 1e-6 along directions whose
  differences no ReLU kink spoils, 1e-3 along a random-sign table direction (kink-limited).

Targets: the oracle's rendering of the seeded scene at the batch's pixels, written into
full-image crops (zero elsewhere: only the batch's pixels are read)."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import render, step as OS, targets as OT
from synth import unpack_pixel, workloads as W
from gpu_util import (GRAD_REL_MIXED, MAX_FLIPS, RGB_REL_MIXED, Case, close, explain_with_flips, flip_groups,
                      mask_flip_deltas, model_config, normwise)

pytestmark = pytest.mark.gpu
N_RAYS = 4096
SEED = 5  # sampler seed of the step (training jitter), the oracle's too


def sparse_targets(w, cams, pix):
    """Per-view full-image crops holding the oracle's target colour at the batch's pixels."""
    hf = W.scene(w)
    top, d = OT.rays_fp64(cams, pix, np.zeros(3), hf.lo[2], hf.hi[2])
    col = OT.shade_rays(hf, top, d)
    v, r, c = unpack_pixel(pix)
    imgs = []
    for vi, cam in enumerate(cams):
        r0, c0, h, wd = cam.crop
        img = np.zeros((h, wd, 3), np.float32)
        m = v == vi
        img[r[m] - r0, c[m] - c0] = col[m]
        imgs.append(img)
    return imgs


def headline_case(name):
    w = dataclasses.replace(W.get(name), n_rays=N_RAYS)
    cams = W.cameras(w)
    pix = W.batch(w, cams, 77)
    cfg = model_config(w)
    lay = cfg.grid()
    params = W.init_params(lay.n_params, cfg.geo_shapes(), cfg.col_shapes(), cfg.n_slots, cfg.n_colour_blocks(), 0)
    rng = np.random.default_rng(9)
    for a, b, mlp_a in OS.group_ranges(cfg)[:cfg.n_slots]:
        params[a:mlp_a] = rng.uniform(-0.3, 0.3, mlp_a - a).astype(np.float32)  # a non-trivial field
    return Case(w, cams, sparse_targets(w, cams, pix), cfg, params, pix)


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def gpu_step(ctx, case):
    w = case.w
    crops = [torch.from_numpy(t).cuda() for t in case.targets]
    ctx.set_views(case.cams, crops)
    tr = Trainer(ctx, model_from_workload(w, snk.SNK_MIXED), snk.window_struct(w.window()),
                 snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, SEED, 0), case.params)
    out = torch.zeros(N_RAYS * 5, dtype=torch.float32, device="cuda")
    tr.train_step(torch.from_numpy(case.pix.view(np.int32)).cuda(), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    res = dict(state=tr.read_state(), out=out.cpu().numpy().reshape(N_RAYS, 5),
               m=tr.m.cpu().numpy().astype(np.float64), adam=tr.adam)
    del tr, crops
    torch.cuda.empty_cache()
    return res


def oracle_step(case):
    n = len(case.params)
    wc = case.params.astype(np.float16).astype(np.float64)  # the working copy the GPU computes with
    ref = OS.train_step(case.cfg, wc, np.zeros(n), np.zeros(n), [0] * case.cfg.n_optimisers(), case.cams,
                        case.w.window(), case.pix, case.targets, SEED, 0)
    return wc, ref


def check_against_oracle(case, got, wc, ref):
    st = got["state"]
    assert st["n_samples"] == int(ref.seg.ray_off[-1]) and st["n_accepted"] == int(ref.seg.ray_ok.sum())
    assert st["n_samples"] > 300_000
    go = got["out"]
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a, b, RGB_REL_MIXED)
        assert ok, (nm, err)
    m = got["m"]
    deltas = mask_flip_deltas(case, ref, wc)
    ref_m, flips = explain_with_flips(m, ref.m, [(1.0 - 0.9) * d for d in deltas], flip_groups(case.cfg))
    print("%s: %d samples, ambiguous ReLU decisions %d, accepted flips %d %s"
          % (case.w.name, st["n_samples"], len(deltas), len(flips), ["%.2e" % f for f in flips]))
    assert len(flips) <= MAX_FLIPS, flips
    errs, elem = {}, {}
    lay = case.cfg.grid()
    for gi, (a, b, mlp_a) in enumerate(OS.group_ranges(case.cfg)):
        if mlp_a > a:
            errs["table%d" % gi] = normwise(m[a:mlp_a], ref_m[a:mlp_a])
        errs["mlp%d" % gi] = normwise(m[mlp_a:b], ref_m[mlp_a:b])
        # the MLP matrices element by element
        shapes = case.cfg.geo_shapes() if gi < case.cfg.n_slots else case.cfg.col_shapes()
        p = mlp_a
        for k, (r, c) in enumerate(shapes):
            ok, err = close(m[p:p + r * c], ref_m[p:p + r * c], GRAD_REL_MIXED)
            elem["g%d.W%d" % (gi, k + 1)] = err / max(np.abs(ref_m[p:p + r * c]).max(), 1e-300)
            assert ok, ("group %d matrix %d" % (gi, k + 1), err)
            p += r * c
    print("%s gradient errors (norm-wise): %s" % (case.w.name, {k: "%.2e" % v for k, v in errs.items()}))
    print("%s MLP max element errors (rel. to max): %s" % (case.w.name, {k: "%.2e" % v for k, v in elem.items()}))
    assert max(errs.values()) < GRAD_REL_MIXED, errs
    assert lay.n_entries > 6_000_000
    return ref_m


def test_window2x2_full_model_gradients_match_the_oracle(ctx):
    case = headline_case("window2x2_full")
    got = gpu_step(ctx, case)
    wc, ref = oracle_step(case)
    check_against_oracle(case, got, wc, ref)


def test_tile512_full_model_gradients_match_the_oracle_and_central_differences(ctx):
    case = headline_case("tile512_full")
    got = gpu_step(ctx, case)
    wc, ref = oracle_step(case)
    check_against_oracle(case, got, wc, ref)
    cfg = case.cfg
    # central differences of the oracle's loss along random directions, the samples held fixed
    # (parameters move no sample: the positions come from the cameras and the sampler)
    smp, seg, gt = ref.smp, ref.seg, ref.extra["gt"]
    t, dt = smp.t.astype(np.float64), smp.dt.astype(np.float64)

    def loss(flat):
        sigma, rgb_s, _ = OS.field_forward(cfg, flat, smp, dirs=ref.extra["d"])
        rgb = render.composite(sigma, rgb_s, t, dt, seg.ray_off)[0]
        return render.mse_loss(rgb, gt, seg.ray_ok)[0]

    assert abs(loss(wc) - ref.loss) <= 1e-12 * ref.loss
    # the GPU's gradient: Adam's first moment is (1 - beta1) (g + l2 w) on MLP weights, (1 - beta1) g on tables
    a, b, mlp_a = OS.group_ranges(cfg)[0]
    ca, cb, _ = OS.group_ranges(cfg)[1]
    g_gpu = got["m"] / (1.0 - got["adam"].beta1)
    l2 = np.zeros_like(wc)
    l2[mlp_a:b] = got["adam"].l2_mlp
    l2[ca:cb] = got["adam"].l2_mlp
    g_gpu = g_gpu - l2 * case.params.astype(np.float64)  # the decay acts on the binary32 master weights
    # Directions, steps and the oracle's tolerance.  A direction through the ReLUs crosses a few
    # kinks at any step, each spoiling the difference by up to half its unit's own term; a
    # coherent direction (every term of g.v positive) or a tiny step keeps that far below the
    # tolerance, while a random-sign direction of the table, whose derivative is a cancelling sum,
    # is kink-limited to ~2e-4 (measured at h = 1e-7: larger steps cross more kinks, smaller ones
    # meet FP64 rounding).  The colour output layer has no ReLU after it: exact to rounding.
    rng = np.random.default_rng(21)
    geo, col = cfg.geo_shapes(), cfg.col_shapes()
    v3 = ca + col[0][0] * col[0][1] + col[1][0] * col[1][1]
    table = np.arange(a, mlp_a)
    cases = [("table, coherent", table, np.sign(ref.grad[a:mlp_a]) * rng.uniform(0.5, 1.0, mlp_a - a), 1e-8, 1e-6),
             ("table, random signs", table, rng.standard_normal(mlp_a - a), 1e-7, 1e-3),
             ("density MLP", np.arange(mlp_a, b), rng.standard_normal(b - mlp_a), 1e-8, 2e-6),
             ("colour MLP", np.arange(ca, cb), rng.standard_normal(cb - ca), 1e-8, 2e-6),
             ("colour output layer", np.arange(v3, cb), rng.standard_normal(cb - v3), 1e-6, 1e-6)]
    for nm, idx, vals, step, tol in cases:
        v = np.zeros_like(wc)
        v[idx] = vals
        h = step / np.abs(v).max()
        fd = (loss(wc + h * v) - loss(wc - h * v)) / (2 * h)
        an = float(ref.grad @ v)
        gp = float(g_gpu @ v)
        print("%s: FD %.9e, oracle %.9e (rel %.1e), GPU %.9e (rel %.1e)"
              % (nm, fd, an, abs(an - fd) / abs(fd), gp, abs(gp - fd) / abs(fd)))
        assert abs(an - fd) <= tol * abs(fd), (nm, an, fd)
        assert abs(gp - fd) <= GRAD_REL_MIXED * abs(fd), (nm, gp, fd)
