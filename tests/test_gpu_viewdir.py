"""View-direction colour input (the colour network on [g | SH_16(d)], degrees
0..3 of the ray direction as in Instant-NGP's direction encoding) on the
device against the oracle: a training step and a render on the binary32 and
the mixed path within their tolerances, and the exact reduction to the model
without directions when the direction weights are zero."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import step as OS
from gpu_util import GRAD_REL_FP32, GRAD_REL_MIXED, RGB_REL_FP32, RGB_REL_MIXED, close, make_case, normwise
from test_gpu_mixed import working_copy
from gpu_util import MAX_FLIPS, explain_with_flips, flip_groups, mask_flip_deltas

pytestmark = pytest.mark.gpu
NAME = "tiny_window_vd"


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _trainer(ctx, case, precision, params=None, render=0, w=None):
    w = w or case.w
    crops = [dev(t.astype(np.float32)) for t in case.targets] if case.targets is not None else None
    ctx.set_views(case.cams, crops)
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, render, 5, 0)
    tr = Trainer(ctx, model_from_workload(w, precision), snk.window_struct(w.window()), sp,
                 case.params if params is None else params)
    tr._crops = crops
    return tr


@pytest.mark.parametrize("precision", [snk.SNK_FP32, snk.SNK_MIXED])
@pytest.mark.parametrize("n_rays", [160, 700])
def test_train_step_with_view_directions_matches_oracle(ctx, precision, n_rays):
    case = make_case(NAME, n_rays=n_rays, table_scale=0.3)
    assert case.cfg.view_dirs and case.cfg.col_shapes()[0] == (64, case.w.geo_out + 16)
    tr = _trainer(ctx, case, precision)
    out = torch.zeros(n_rays * 5, dtype=torch.float32, device="cuda")
    tr.train_step(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    n = len(case.params)
    mixed = precision != snk.SNK_FP32
    wc = working_copy(case.params, case.cfg) if mixed else case.params.astype(np.float64)
    ref = OS.train_step(case.cfg, wc, np.zeros(n), np.zeros(n), [0] * case.cfg.n_optimisers(), case.cams,
                        case.w.window(), case.pix, case.targets, 5, 0)
    assert tr.read_state()["n_samples"] == int(ref.seg.ray_off[-1])
    go = out.cpu().numpy().reshape(n_rays, 5)
    tol = RGB_REL_MIXED if mixed else RGB_REL_FP32
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a, b, tol)
        assert ok, (nm, err)
    m = tr.m.cpu().numpy().astype(np.float64)
    ref_m = ref.m
    if mixed:
        ref_m, flips = explain_with_flips(m, ref.m, [(1.0 - 0.9) * d for d in mask_flip_deltas(case, ref, wc)],
                                         flip_groups(case.cfg))
        print("accepted flips: %d %s" % (len(flips), ["%.2e" % f for f in flips]))
        assert len(flips) <= MAX_FLIPS, flips
    errs = {}
    for gi, (a, b, mlp_a) in enumerate(OS.group_ranges(case.cfg)):
        if mlp_a > a:
            errs["table%d" % gi] = normwise(m[a:mlp_a], ref_m[a:mlp_a])
        errs["mlp%d" % gi] = normwise(m[mlp_a:b], ref_m[mlp_a:b])
    print("gradient errors (norm-wise):", errs)
    assert max(errs.values()) < (GRAD_REL_MIXED if mixed else GRAD_REL_FP32), errs
    # the direction columns of V1 receive a gradient
    _, cols = OS.unflatten(case.cfg, m)
    assert np.abs(cols[0][0][:, case.w.geo_out:]).max() > 0


@pytest.mark.parametrize("precision", [snk.SNK_FP32, snk.SNK_MIXED])
def test_render_with_view_directions_matches_oracle(ctx, precision):
    case = make_case(NAME, n_rays=500, table_scale=0.3, with_targets=False)
    tr = _trainer(ctx, case, precision, render=1)
    out = torch.zeros(500 * 5, dtype=torch.float32, device="cuda")
    tr.render(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    mixed = precision != snk.SNK_FP32
    wc = working_copy(case.params, case.cfg) if mixed else case.params.astype(np.float64)
    ref = OS.render_rays(case.cfg, wc, case.cams, case.w.window(), case.pix)
    go = out.cpu().numpy().reshape(500, 5)
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a, b, RGB_REL_MIXED if mixed else RGB_REL_FP32)
        assert ok, (nm, err)


@pytest.mark.parametrize("precision", [snk.SNK_FP32, snk.SNK_MIXED])
def test_zero_direction_weights_reduce_to_the_model_without_directions(ctx, precision):
    """With the direction columns of V1 at zero the colour input's extra terms
    add exact zeros: the render equals the plain model's, and a step's
    gradients of every parameter the plain model has are the plain model's."""
    case = make_case(NAME, n_rays=300, table_scale=0.3)
    cfg_vd = case.cfg
    cfg_0 = dataclasses.replace(cfg_vd, view_dirs=False)
    w0 = dataclasses.replace(case.w, view_dirs=False)
    G = case.w.geo_out
    # plain parameters: the VD case's with V1 cut to its g columns
    t_vd, c_vd = OS.unflatten(cfg_vd, case.params)
    flat0 = np.zeros(cfg_0.n_params(), np.float32)
    t0, c0 = OS.unflatten(cfg_0, flat0)
    for k in range(cfg_vd.n_slots):
        t0[k][0][...] = t_vd[k][0]
        for q in range(3):
            t0[k][1][q][...] = t_vd[k][1][q]
    for b in range(len(c_vd)):
        c0[b][0][...] = c_vd[b][0][:, :G]
        c_vd[b][0][:, G:] = 0.0  # case.params is modified in place: direction weights zero
        for q in (1, 2):
            c0[b][q][...] = c_vd[b][q]
    pix = dev(case.pix.view(np.int32))
    outs, ms = [], []
    for params, w in [(case.params, case.w), (flat0, w0)]:
        tr = _trainer(ctx, case, precision, params=params, w=w, render=1)
        out = torch.zeros(300 * 5, dtype=torch.float32, device="cuda")
        tr.render(pix, out)
        outs.append(out.cpu().numpy())
        tr = _trainer(ctx, case, precision, params=params, w=w)
        tr.train_step(pix)
        assert ctx.sync_status(tr.state) == snk.SNK_OK
        ms.append(tr.m.cpu().numpy())
    if precision == snk.SNK_FP32:
        assert np.array_equal(outs[0], outs[1])
    else:
        assert np.allclose(outs[0], outs[1], rtol=1e-6, atol=1e-7)
    m_vd = OS.unflatten(cfg_vd, ms[0])
    m_0 = OS.unflatten(cfg_0, ms[1])
    pairs = [(m_vd[0][k][0], m_0[0][k][0]) for k in range(cfg_vd.n_slots)]
    pairs += [(m_vd[0][k][1][q], m_0[0][k][1][q]) for k in range(cfg_vd.n_slots) for q in range(3)]
    pairs += [(m_vd[1][b][0][:, :G], m_0[1][b][0]) for b in range(len(c_vd))]
    pairs += [(m_vd[1][b][q], m_0[1][b][q]) for b in range(len(c_vd)) for q in (1, 2)]
    for a, b in pairs:
        # the same sums in the same order, except the scatter's atomic order (tables) and flushes
        assert normwise(a.astype(np.float64), b.astype(np.float64)) < 1e-6



def test_stored_and_recomputed_activations_agree(ctx):
    """Mixed path with view directions: the backward reading the stored activations
    and the backward recomputing them compute the same step."""
    case = make_case(NAME, n_rays=300, table_scale=0.3)
    ms = []
    for saved in (1, 0):
        ctx.set_tuning(tc_bwd_saved=saved)
        tr = _trainer(ctx, case, snk.SNK_MIXED)
        out = torch.zeros(300 * 5, dtype=torch.float32, device="cuda")
        tr.train_step(dev(case.pix.view(np.int32)), out)
        assert ctx.sync_status(tr.state) == snk.SNK_OK
        ms.append((out.cpu().numpy(), tr.m.cpu().numpy().astype(np.float64)))
    ctx.set_tuning(tc_bwd_saved=1)
    assert np.array_equal(ms[0][0], ms[1][0])
    assert normwise(ms[0][1], ms[1][1]) < 1e-5
