"""Sampler variants on the device against the oracle: the NeRF-XL uniform
distribution and point samples with backward-difference deltas, bit-exact
(segments, counts, sample positions, deltas) in training and rendering, and a
binary32 training step in each mode within the binary32 tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import sampler as OSM, step as OS
from gpu_util import GRAD_REL_FP32, RGB_REL_FP32, close, gpu_sample, gpu_to_ray_major, make_case, normwise

pytestmark = pytest.mark.gpu
MODES = [(snk.SNK_SAMPLE_UNIFORM, OSM.UNIFORM), (snk.SNK_SAMPLE_POINTS, OSM.POINTS)]


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("mode,omode", MODES)
@pytest.mark.parametrize("name,n_rays", [("tiny_window", 160), ("window2x2_full", 600), ("tile512_full", 200)])
@pytest.mark.parametrize("render", [0, 1])
def test_sampling_modes_are_bit_exact(ctx, mode, omode, name, n_rays, render):
    case = make_case(name, n_rays=n_rays, with_targets=False)
    w = case.w
    ctx.set_views(case.cams)
    K_min = max(w.K_min, 2)
    sp = snk.sampler_struct(w.K_ray, K_min, w.K_max, render, 7, 3, mode=mode)
    h = gpu_sample(ctx, case, sp)
    cfg = case.cfg
    cfg.K_min = K_min
    _, _, seg, smp = OS.sample_rays(cfg, case.cams, w.window(), case.pix, 7, 3, bool(render), mode=omode)
    B = n_rays
    assert np.array_equal(h["ray_ok"], seg.ray_ok)
    assert np.array_equal(h["seg_slot"].reshape(B, 3).astype(np.int64), seg.slot)
    seg_t = h["seg_t"].reshape(B, 3, 2)
    assert np.array_equal(seg_t[..., 0], seg.t0) and np.array_equal(seg_t[..., 1], seg.t1)
    assert np.array_equal(h["seg_n"].reshape(B, 3), seg.K)
    assert h["n_samples"] == int(seg.ray_off[-1])
    idx = gpu_to_ray_major(h["seg_n"].reshape(B, 3), h["seg_off"].reshape(B, 3), seg.ray_off)
    assert np.array_equal(h["smp_t"][idx], smp.t) and np.array_equal(h["smp_dt"][idx], smp.dt)
    assert np.array_equal(h["smp_xyz"].reshape(-1, 3)[idx], smp.xyz)


@pytest.mark.parametrize("mode,omode", MODES)
def test_train_step_in_each_mode_matches_oracle(ctx, mode, omode):
    case = make_case("tiny_window", n_rays=160, table_scale=0.3)
    w = case.w
    crops = [torch.from_numpy(t.astype(np.float32)).cuda() for t in case.targets]
    ctx.set_views(case.cams, crops)
    sp = snk.sampler_struct(w.K_ray, max(w.K_min, 2), w.K_max, 0, 5, 0, mode=mode)
    tr = Trainer(ctx, model_from_workload(w, snk.SNK_FP32), snk.window_struct(w.window()), sp, case.params)
    out = torch.zeros(160 * 5, dtype=torch.float32, device="cuda")
    tr.train_step(torch.from_numpy(case.pix.view(np.int32)).cuda(), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    cfg = case.cfg
    cfg.K_min = max(w.K_min, 2)
    n = len(case.params)
    ref = OS.train_step(cfg, case.params.astype(np.float64), np.zeros(n), np.zeros(n), [0] * cfg.n_optimisers(),
                        case.cams, w.window(), case.pix, case.targets, 5, 0, mode=omode)
    go = out.cpu().numpy().reshape(160, 5)
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        good, err = close(a, b, RGB_REL_FP32)
        assert good, (nm, err)
    m = tr.m.cpu().numpy().astype(np.float64)
    for a, b, mlp_a in OS.group_ranges(cfg):
        assert normwise(m[a:b], ref.m[a:b]) < GRAD_REL_FP32


def test_invalid_mode_combinations_are_rejected(ctx):
    case = make_case("tiny_window", n_rays=8, with_targets=False)
    w = case.w
    ctx.set_views(case.cams)
    occ = torch.ones(4 * 16 ** 3, dtype=torch.uint8, device="cuda")
    for sp in [snk.sampler_struct(w.K_ray, w.K_min, w.K_max, mode=3),
               snk.sampler_struct(w.K_ray, 1, w.K_max, mode=snk.SNK_SAMPLE_POINTS),
               snk.sampler_struct(w.K_ray, w.K_min, w.K_max, mode=snk.SNK_SAMPLE_UNIFORM, occupancy=occ, occ_res=16)]:
        with pytest.raises(RuntimeError):
            gpu_sample(ctx, case, sp)
