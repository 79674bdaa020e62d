"""Mixed-precision path (FP16 tables, FP16 MLP on the tcgen05 tensor cores, FP32
accumulation, loss scaling) against the FP64 oracle, through the C ABI.

The oracle runs on the parameters the mixed model computes with: its FP16
working copy.  Tolerances: rendered RGB
and depth rel 2e-3 (floor 2e-3 x max), gradients 5e-3 norm-wise per tensor."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import step as OS
from gpu_util import GRAD_REL_MIXED, MAX_FLIPS, RGB_REL_MIXED, close, explain_with_flips, flip_groups, \
    make_case, mask_flip_deltas, normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def working_copy(params, cfg):
    """FP64 values of the mixed model's working copy of binary32 parameters."""
    return params.astype(np.float16).astype(np.float64)


def _trainer(ctx, case, seed=5, render=0):
    w = case.w
    crops = [dev(t.astype(np.float32)) for t in case.targets] if case.targets is not None else None
    ctx.set_views(case.cams, crops)
    model = model_from_workload(w, snk.SNK_MIXED)
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, render, seed, 0)
    tr = Trainer(ctx, model, snk.window_struct(w.window()), sp, case.params)
    tr._crops = crops
    return tr


MIXED_CASES = [("tiny_tile", 96, None), ("tiny_window", 160, None), ("tile256_fp32", 512, None),
               ("tile512_full", 512, 48), ("window2x2_full", 512, 48)]


def check_step_against_oracle(case, tr, out):
    """The first mixed step of `tr` (rendered `out`) against the FP64 oracle on the working copy:
    rendered rays, loss, every parameter group's gradient (via Adam's first moment) with the
    ambiguous-ReLU flips accounted for, the first Adam move, the refreshed working copy."""
    B = len(case.pix)
    st = tr.read_state()
    n = len(case.params)
    wc = working_copy(case.params, case.cfg)
    ref = OS.train_step(case.cfg, wc, np.zeros(n), np.zeros(n), [0] * case.cfg.n_optimisers(), case.cams,
                        case.w.window(), case.pix, case.targets, 5, 0)
    assert st["n_samples"] == int(ref.seg.ray_off[-1]) and st["n_accepted"] == int(ref.seg.ray_ok.sum())
    go = out.cpu().numpy().reshape(B, 5)
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a, b, RGB_REL_MIXED)
        assert ok, (nm, err)
    # loss = mean (C - gt)^2: an RGB error e changes it by at most 2 sqrt(loss) e
    e = RGB_REL_MIXED * 2 * max(1.0, np.abs(ref.rgb).max())
    assert abs(st["loss"] - ref.loss) <= 2 * np.sqrt(ref.loss) * e + 1e-7, (st["loss"], ref.loss)
    m = tr.m.cpu().numpy().astype(np.float64)
    # decisions that may legitimately differ: account for flipped near-zero ReLU masks
    deltas = mask_flip_deltas(case, ref, wc)
    ref_m, flips = explain_with_flips(m, ref.m, [(1.0 - 0.9) * d for d in deltas], flip_groups(case.cfg))
    print("ambiguous ReLU decisions: %d, accepted flips: %d, their sizes relative to |m|: %s"
          % (len(deltas), len(flips), ["%.2e" % f for f in flips]))
    assert len(flips) <= MAX_FLIPS, flips
    errs = {}
    for gi, (a, b, mlp_a) in enumerate(OS.group_ranges(case.cfg)):
        if mlp_a > a:
            errs["table%d" % gi] = normwise(m[a:mlp_a], ref_m[a:mlp_a])
        errs["mlp%d" % gi] = normwise(m[mlp_a:b], ref_m[mlp_a:b])
    print("gradient errors (norm-wise):", errs)
    assert max(errs.values()) < GRAD_REL_MIXED, errs
    for gi, (a, b, mlp_a) in enumerate(OS.group_ranges(case.cfg)):
        # parameters with a clearly non-zero gradient move by the oracle's first Adam step
        pg = tr.params.cpu().numpy().astype(np.float64)[a:b]
        moved = ref.params[a:b] - wc[a:b]
        rg = np.abs(ref.grad[a:b])
        sure = rg > 5e-2 * max(rg.max(), 1e-30)
        assert np.allclose(pg[sure], case.params[a:b][sure] + moved[sure], rtol=0, atol=1e-5)
    assert np.all(tr.steps.cpu().numpy() == 1)
    assert np.all(tr.grads.cpu().numpy() == 0)
    # the working copy was refreshed from the updated master weights
    lp = tr.params_lp.cpu()
    assert torch.equal(lp, tr.params.cpu().to(torch.float16).view(torch.int16))
    return st


@pytest.mark.parametrize("name,n_rays,crop", MIXED_CASES)
def test_train_step_mixed_matches_oracle(ctx, name, n_rays, crop):
    case = make_case(name, n_rays=n_rays, crop=crop, table_scale=0.3)
    tr = _trainer(ctx, case)
    out = torch.zeros(n_rays * 5, dtype=torch.float32, device="cuda")
    tr.train_step(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    check_step_against_oracle(case, tr, out)


def test_activation_budget_switches_the_step_to_recompute(ctx):
    """A budget smaller than the stored-activation buffer makes the step recompute the
    activations in its backward instead of failing: the state reports the mode, the step
    matches the oracle, and it computes what the stored mode computes (rendered outputs bit
    for bit, moments up to the order of float atomics)."""
    case = make_case("tile512_full", n_rays=512, crop=48, table_scale=0.3)
    runs = {}
    try:
        for budget in (None, 4096):
            ctx.set_act_budget(budget)
            tr = _trainer(ctx, case)
            out = torch.zeros(512 * 5, dtype=torch.float32, device="cuda")
            tr.train_step(dev(case.pix.view(np.int32)), out)
            assert ctx.sync_status(tr.state) == snk.SNK_OK
            runs[budget] = (tr, out)
    finally:
        ctx.set_act_budget(None)
    assert runs[None][0].read_state()["bwd_mode"] == 1
    assert runs[4096][0].read_state()["bwd_mode"] == 2
    assert torch.equal(runs[None][1], runs[4096][1])
    assert normwise(runs[4096][0].m.cpu().numpy().astype(np.float64),
                    runs[None][0].m.cpu().numpy().astype(np.float64)) < 1e-5
    check_step_against_oracle(case, *runs[4096])


def test_working_copy_is_written_by_the_library(ctx):
    """snk_params_refresh_lp (called by the trainer) rounds every master weight to the nearest
    FP16, ties to even, as torch's IEEE conversion does, including ties, overflow and
    subnormals."""
    case = make_case("tiny_window", n_rays=8, table_scale=0.3, with_targets=False)
    params = case.params.copy()
    special = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -(1 + 2.0 ** -11), 65504.0, 65520.0, -65536.0,
                        2.0 ** -25, 3 * 2.0 ** -26, 1e-8, 2.0 ** -14, 0.0, -0.0], np.float32)
    params[:len(special)] = special
    case.params = params
    tr = _trainer(ctx, case)
    torch.cuda.synchronize()
    want = torch.from_numpy(params).to(torch.float16).view(torch.int16)
    assert torch.equal(tr.params_lp.cpu(), want)
    assert tr.read_state()["bwd_mode"] == 0  # no step yet


@pytest.mark.parametrize("name,n_rays", [("tiny_window", 160), ("tile512_full", 400), ("window2x2_full", 600)])
def test_render_mixed_matches_oracle(ctx, name, n_rays):
    case = make_case(name, n_rays=n_rays, table_scale=0.3, with_targets=False)
    tr = _trainer(ctx, case, render=1)
    out = torch.zeros(n_rays * 5, dtype=torch.float32, device="cuda")
    tr.render(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    ref = OS.render_rays(case.cfg, working_copy(case.params, case.cfg), case.cams, case.w.window(), case.pix)
    go = out.cpu().numpy().reshape(n_rays, 5)
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a, b, RGB_REL_MIXED)
        assert ok, (nm, err)


def test_mixed_training_reduces_the_loss_and_skips_overflow_steps(ctx):
    """Twenty mixed steps on a window: finite, decreasing loss.  A non-finite
    value injected from the host into the gradient accumulator makes the next
    step skip its update (status bit 0), halve the loss scale, leave the
    weights unchanged and clear the accumulator."""
    case = make_case("tiny_window", n_rays=160, table_scale=1e-4)
    tr = _trainer(ctx, case)
    pix = dev(case.pix.view(np.int32))
    losses = []
    for i in range(20):
        tr.train_step(pix)
        losses.append(tr.read_state()["loss"])
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]
    before = tr.params.clone()
    scale = tr.read_state()["loss_scale"]
    steps = tr.steps.clone()
    tr.grads[123] = float("nan")
    tr.train_step(pix)
    st = tr.read_state()
    assert st["status"] & snk.STATUS_OVERFLOW
    assert st["loss_scale"] == pytest.approx(scale / 2, rel=1e-6)
    assert torch.equal(tr.params, before) and torch.equal(tr.steps, steps)
    assert torch.count_nonzero(tr.grads) == 0
    assert ctx.sync_status(tr.state) == snk.SNK_ERR_OVERFLOW
