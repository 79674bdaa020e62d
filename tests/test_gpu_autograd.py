"""The torch.autograd.Function wrappers (SnkEncode -> SnkMLP -> SnkComposite)
composed by PyTorch's autograd, against the FP64 oracle's analytic gradient of
the same step: loss = mean over accepted rays and channels of (C - C_gt)^2.

Tolerances as for the binary32 path: rendered RGB rel 1e-5, gradients 5e-4
norm-wise per parameter group (tables of a slot, MLP weights of a slot,
colour net)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.autograd import SnkComposite, SnkEncode, SnkMLP, Stages
from paper_2507_01631_b300.trainer import model_from_workload
from oracle import step as OS
import synth
from gpu_util import GRAD_REL_FP32, RGB_REL_FP32, close, make_case, normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def targets_of(case):
    """Target colour of every ray, read from its view's crop (test-side gather)."""
    v, r, c = synth.unpack_pixel(case.pix)
    gt = np.zeros((len(v), 3), np.float32)
    for i in range(len(v)):
        r0, c0, _, _ = case.cams[v[i]].crop
        gt[i] = case.targets[v[i]][r[i] - r0, c[i] - c0]
    return gt


@pytest.mark.parametrize("name,n_rays,crop", [("tiny_tile", 96, None), ("tiny_window", 160, None),
                                              ("tile256_fp32", 512, None), ("window2x2_full", 400, 48)])
def test_autograd_step_matches_oracle_gradient(ctx, name, n_rays, crop):
    case = make_case(name, n_rays=n_rays, crop=crop, table_scale=0.3)
    w = case.w
    ctx.set_views(case.cams)
    st = Stages(ctx, model_from_workload(w, snk.SNK_FP32), snk.window_struct(w.window()))
    sampler = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 5, 0)
    pix = torch.from_numpy(case.pix.view(np.int32)).cuda()
    batch = st.sample(pix, sampler)
    params = torch.from_numpy(case.params).cuda().requires_grad_(True)
    rgb, depth, opacity = st.render(params, batch)
    assert not depth.requires_grad and not opacity.requires_grad
    gt = torch.from_numpy(targets_of(case)).cuda()
    ok = batch.ray_ok.bool()
    loss = ((rgb - gt) ** 2)[ok].sum() / (3 * ok.sum())
    loss.backward()
    torch.cuda.synchronize()

    n = len(case.params)
    ref = OS.train_step(case.cfg, case.params.astype(np.float64), np.zeros(n), np.zeros(n),
                        [0] * case.cfg.n_optimisers(), case.cams, w.window(), case.pix, case.targets, 5, 0)
    assert np.array_equal(batch.ray_ok.cpu().numpy(), ref.seg.ray_ok)
    for nm, a, b in [("rgb", rgb.detach().cpu().numpy(), ref.rgb), ("depth", depth.cpu().numpy(), ref.depth),
                     ("opacity", opacity.cpu().numpy(), ref.opacity)]:
        good, err = close(a, b, RGB_REL_FP32)
        assert good, (nm, err)
    good, err = close([float(loss)], [ref.loss], RGB_REL_FP32)
    assert good, ("loss", float(loss), ref.loss)
    g = params.grad.cpu().numpy().astype(np.float64)
    for gi, (a, b, mlp_a) in enumerate(OS.group_ranges(case.cfg)):
        if mlp_a > a:
            assert normwise(g[a:mlp_a], ref.grad[a:mlp_a]) < GRAD_REL_FP32, ("table", gi)
        assert normwise(g[mlp_a:b], ref.grad[mlp_a:b]) < GRAD_REL_FP32, ("mlp", gi)


def test_autograd_gradient_is_linear_and_depth_is_not_differentiable(ctx):
    """Doubling the upstream gradient doubles every parameter gradient (up to
    the order of float atomics); depth and opacity carry no gradient."""
    case = make_case("tiny_window", n_rays=96, table_scale=0.3, with_targets=False)
    w = case.w
    ctx.set_views(case.cams)
    st = Stages(ctx, model_from_workload(w, snk.SNK_FP32), snk.window_struct(w.window()))
    batch = st.sample(torch.from_numpy(case.pix.view(np.int32)).cuda(),
                      snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 1, 0, 0))
    grads = []
    for scale in (1.0, 2.0):
        params = torch.from_numpy(case.params).cuda().requires_grad_(True)
        rgb, depth, opacity = st.render(params, batch)
        (scale * (rgb * rgb).sum()).backward()
        grads.append(params.grad.double().cpu().numpy())
    assert np.count_nonzero(grads[0]) > 0
    assert normwise(grads[1], 2.0 * grads[0]) < 1e-6
    params = torch.from_numpy(case.params).cuda().requires_grad_(True)
    rgb, depth, opacity = st.render(params, batch)
    with pytest.raises(RuntimeError):
        (depth.sum() + opacity.sum()).backward()
