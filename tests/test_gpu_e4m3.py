"""Mixed-precision stress configuration: E4M3 first-layer input with a
per-slot scale from the current batch (SNK_MIXED_E4M3), on the raster-blocks
scene with long slant segments, against the FP64 oracle taking the same
quantisation decisions (oracle/quant.py).

The quantiser itself is bit-exact (a conversion of exactly representable
inputs).  In the training step both sides decide the codes in binary32 (the
oracle from a binary32 replica of the kernel's features); a code decided
within two binary32 ulps of a tie between two E4M3 values may still go either
way, so rays holding one are left out of the element-wise comparison (their
share is bounded) and the gradients are compared norm-wise at the mixed
tolerances.  The tests
also print the error of the quantised path against the unquantised FP64
oracle: the price of the 8-bit input."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import hashgrid, quant, step as OS
from gpu_util import GRAD_REL_MIXED, RGB_REL_MIXED, close, make_case, normwise

pytestmark = pytest.mark.gpu
TIE_WINDOW = 2.0 ** -22  # two binary32 ulps: a code decided this close to a tie may still differ


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_quantizer_bit_exact(ctx):
    rng = np.random.default_rng(0)
    vals = np.sort(quant.e4m3_decode(np.arange(0, 0x7F, dtype=np.uint8)))
    ties = 0.5 * (vals[1:] + vals[:-1])
    x = np.concatenate([rng.normal(0, 1, 50000), rng.normal(0, 100, 50000), rng.uniform(-2.0 ** -6, 2.0 ** -6, 50000),
                        ties, -ties, vals, -vals, [0.0, -0.0, 448.0, 463.9, 464.0, 1e6, -1e30]]).astype(np.float32)
    x = np.concatenate([x, x[:7]])  # odd length: the last pair is half full
    for scale in (1.0, 2.0 ** -5, 8.0):
        codes = torch.zeros(len(x), dtype=torch.uint8, device="cuda")
        ctx.call("snk_quantize_e4m3", snk.ptr(dev(x)), len(x), float(scale), snk.ptr(codes), None)
        torch.cuda.synchronize()
        want = quant.e4m3_encode(x.astype(np.float64) / scale)  # x / scale is exact in both precisions
        got = codes.cpu().numpy()
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (scale, x[bad[:5]], got[bad[:5]], want[bad[:5]])
    with pytest.raises(RuntimeError):
        ctx.call("snk_quantize_e4m3", None, 4, 0.0, None, None)


def _ambiguous_rays(case, flat, ref):
    """Rays holding a code decision within two binary32 ulps of an E4M3 tie.
    The oracle decides codes from a binary32 replica of the kernel's features
    (quant.encode_binary32); only such near-ties may still differ."""
    cfg, smp = case.cfg, ref.smp
    tiles, _ = OS.unflatten(cfg, flat)
    lay = cfg.grid()
    vals = np.sort(quant.e4m3_decode(np.arange(0, 0x7F, dtype=np.uint8)))
    ties = 0.5 * (vals[1:] + vals[:-1])
    flag = np.zeros(len(smp.t), bool)
    for k in range(cfg.n_slots):
        m = np.flatnonzero(smp.slot == k)
        if m.size == 0:
            continue
        f32 = quant.encode_binary32(smp.xyz[m], tiles[k][0], lay)
        x = np.abs((f32 / quant.slot_scale_binary32(f32)).astype(np.float32)).astype(np.float64)
        j = np.clip(np.searchsorted(ties, x), 1, len(ties) - 1)
        d = np.minimum(np.abs(x - ties[j - 1]), np.abs(x - ties[j]))
        flag[m] = (d <= TIE_WINDOW * np.maximum(x, 2.0 ** -126)).any(axis=1)
    off = ref.seg.ray_off
    return np.array([flag[off[i]:off[i + 1]].any() for i in range(len(off) - 1)], bool)


def _trainer(ctx, case, seed=5, render=0):
    w = case.w
    crops = [dev(t.astype(np.float32)) for t in case.targets] if case.targets is not None else None
    ctx.set_views(case.cams, crops)
    model = model_from_workload(w, snk.SNK_MIXED_E4M3)
    tr = Trainer(ctx, model, snk.window_struct(w.window()), snk.sampler_struct(w.K_ray, w.K_min, w.K_max, render,
                                                                                seed, 0), case.params)
    tr._crops = crops
    return tr


@pytest.mark.parametrize("name,n_rays,crop", [("tiny_window_fp8", 160, None), ("window2x2_fp8", 384, 48)])
def test_train_step_e4m3_matches_oracle(ctx, name, n_rays, crop):
    case = make_case(name, n_rays=n_rays, crop=crop, table_scale=0.3)
    assert case.cfg.first_layer == "e4m3"
    tr = _trainer(ctx, case)
    B = n_rays
    out = torch.zeros(B * 5, dtype=torch.float32, device="cuda")
    tr.train_step(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    st = tr.read_state()
    n = len(case.params)
    wc = case.params.astype(np.float16).astype(np.float64)  # the working copy the GPU computes with
    args = (np.zeros(n), np.zeros(n), [0] * case.cfg.n_optimisers(), case.cams, case.w.window(), case.pix,
            case.targets, 5, 0)
    ref = OS.train_step(case.cfg, wc, *args)
    assert st["n_samples"] == int(ref.seg.ray_off[-1]) and st["n_accepted"] == int(ref.seg.ray_ok.sum())
    amb = _ambiguous_rays(case, wc, ref)
    print("rays with a feature at an E4M3 tie: %d of %d" % (amb.sum(), B))
    # decided by the oracle alone, so fixed by the seeds: 1 of 160 and 19 of 384 rays (about
    # 6e-6 of the codes fall within two ulps of a tie; a ray of the window holds ~8300 codes)
    assert amb.mean() <= 0.05, amb.sum()
    go = out.cpu().numpy().reshape(B, 5)
    keep = ~amb
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a[keep], b[keep], RGB_REL_MIXED)
        assert ok, (nm, err)
    m = tr.m.cpu().numpy().astype(np.float64)
    errs = {}
    for gi, (a, b, mlp_a) in enumerate(OS.group_ranges(case.cfg)):
        if mlp_a > a:
            errs["table%d" % gi] = normwise(m[a:mlp_a], ref.m[a:mlp_a])
        errs["mlp%d" % gi] = normwise(m[mlp_a:b], ref.m[mlp_a:b])
    print("gradient errors vs the quantised oracle (norm-wise):", errs)
    assert max(errs.values()) < GRAD_REL_MIXED, errs
    # the price of the 8-bit input: against the unquantised FP64 oracle
    plain = OS.train_step(dataclasses.replace(case.cfg, first_layer="f16"), wc, *args)
    q_err = {"rgb": float(np.max(np.abs(go[:, :3] - plain.rgb)) / max(np.abs(plain.rgb).max(), 1e-30)),
             "depth": float(np.max(np.abs(go[:, 3] - plain.depth)) / max(np.abs(plain.depth).max(), 1e-30))}
    for gi, (a, b, mlp_a) in enumerate(OS.group_ranges(case.cfg)):
        q_err["grad%d" % gi] = normwise(m[a:b], plain.m[a:b])
    print("E4M3 path vs the unquantised FP64 oracle:", q_err)
    assert q_err["rgb"] < 0.05 and q_err["depth"] < 0.05


@pytest.mark.parametrize("name,n_rays", [("tiny_window_fp8", 160), ("window2x2_fp8", 400)])
def test_render_e4m3_matches_oracle(ctx, name, n_rays):
    case = make_case(name, n_rays=n_rays, table_scale=0.3, with_targets=False)
    tr = _trainer(ctx, case, render=1)
    out = torch.zeros(n_rays * 5, dtype=torch.float32, device="cuda")
    tr.render(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    wc = case.params.astype(np.float16).astype(np.float64)
    ref = OS.render_rays(case.cfg, wc, case.cams, case.w.window(), case.pix)
    amb = _ambiguous_rays(case, wc, ref)
    assert amb.mean() <= 0.05, amb.sum()  # fixed by the seeds: 0 of 160 and 17 of 400 rays
    go = out.cpu().numpy().reshape(n_rays, 5)
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a[~amb], b[~amb], RGB_REL_MIXED)
        assert ok, (nm, err)


def test_e4m3_training_reduces_the_loss(ctx):
    case = make_case("tiny_window_fp8", n_rays=160, table_scale=1e-4)
    tr = _trainer(ctx, case)
    pix = dev(case.pix.view(np.int32))
    losses = []
    for i in range(20):
        tr.train_step(pix)
        losses.append(tr.read_state()["loss"])
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]


def test_stored_and_recomputed_activations_agree(ctx):
    """The backward reading the forward's stored activations and the backward
    recomputing them compute the same step (moments up to the order of float atomics)."""
    case = make_case("tiny_window_fp8", n_rays=160, table_scale=0.3)
    ms = []
    for saved in (1, 0):
        ctx.set_tuning(tc_bwd_saved=saved)
        tr = _trainer(ctx, case)
        out = torch.zeros(160 * 5, dtype=torch.float32, device="cuda")
        tr.train_step(torch.from_numpy(case.pix.view(np.int32)).cuda(), out)
        assert ctx.sync_status(tr.state) == snk.SNK_OK
        ms.append((out.cpu().numpy(), tr.m.cpu().numpy().astype(np.float64)))
    ctx.set_tuning(tc_bwd_saved=1)
    assert np.array_equal(ms[0][0], ms[1][0])
    assert normwise(ms[0][1], ms[1][1]) < 1e-5
