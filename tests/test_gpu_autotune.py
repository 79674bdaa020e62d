"""Launch shapes (snk_autotune / snk_set_tuning): every shape computes the same
step -- rendered outputs bit-identical, gradients equal up to the order of
float atomics; this includes the backward reading the forward's stored
activations against recomputing them, and the forward with dedicated gather
warps against the one whose threads gather and then run the chain, for every
model variant -- and the autotuner leaves the caller's training state alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from gpu_util import make_case, normwise

pytestmark = pytest.mark.gpu
DEFAULT = dict(tc_fwd_split=1, tc_fwd_ctas=2, tc_fwd_levels=1, tc_bwd_saved=1, fp32_ctas=2, composite_threads=256,
               sampler_threads=256)
# overrides of DEFAULT; the CTAs per SM matter only without the gather split
ALTERNATIVES = [dict(tc_fwd_levels=2), dict(tc_fwd_split=0), dict(tc_fwd_split=0, tc_fwd_ctas=1),
                dict(tc_fwd_split=0, tc_fwd_ctas=3), dict(tc_fwd_split=0, tc_fwd_levels=2),
                dict(tc_fwd_split=0, tc_fwd_ctas=3, tc_fwd_levels=2), dict(tc_bwd_saved=0),
                dict(tc_bwd_saved=0, tc_fwd_split=0), dict(fp32_ctas=1), dict(composite_threads=64),
                dict(composite_threads=512), dict(sampler_threads=128), dict(sampler_threads=512)]


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _step(ctx, case, precision):
    crops = [dev(t.astype(np.float32)) for t in case.targets]
    ctx.set_views(case.cams, crops)
    w = case.w
    tr = Trainer(ctx, model_from_workload(w, precision), snk.window_struct(w.window()),
                 snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 5, 0), case.params)
    out = torch.zeros(len(case.pix) * 5, dtype=torch.float32, device="cuda")
    tr.train_step(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    return out.cpu().numpy(), tr.m.cpu().numpy().astype(np.float64), tr.read_state()["loss"]


@pytest.mark.parametrize("precision", [snk.SNK_MIXED, snk.SNK_FP32])
def test_every_launch_shape_computes_the_same_step(ctx, precision):
    case = make_case("window2x2_full", n_rays=384, crop=48, table_scale=0.3)
    ctx.set_tuning(**DEFAULT)
    out0, m0, loss0 = _step(ctx, case, precision)
    for over in ALTERNATIVES:
        ctx.set_tuning(**dict(DEFAULT, **over))
        out, m, loss = _step(ctx, case, precision)
        assert np.array_equal(out, out0), over
        assert abs(loss - loss0) <= 1e-6 * abs(loss0), over
        assert normwise(m, m0) < 1e-5, over
    ctx.set_tuning(**DEFAULT)


@pytest.mark.parametrize("name", ["tiny_tile", "tile256_fp32", "tiny_window", "tiny_window_vd"])
def test_gather_split_computes_the_same_step_for_every_model_variant(ctx, name):
    """Density-only MLP (G = 4) at 8 and 16 features, colour network at 8 features, view
    directions: the forward with dedicated gather warps against the other forward shapes."""
    case = make_case(name, n_rays=384, crop=48, table_scale=0.3)
    ctx.set_tuning(**DEFAULT)
    out0, m0, loss0 = _step(ctx, case, snk.SNK_MIXED)
    for over in [dict(tc_fwd_levels=2), dict(tc_fwd_split=0), dict(tc_fwd_split=0, tc_fwd_ctas=3),
                 dict(tc_bwd_saved=0, tc_fwd_split=0), dict(tc_bwd_saved=0)]:
        ctx.set_tuning(**dict(DEFAULT, **over))
        out, m, loss = _step(ctx, case, snk.SNK_MIXED)
        assert np.array_equal(out, out0), over
        assert abs(loss - loss0) <= 1e-6 * abs(loss0), over
        assert normwise(m, m0) < 1e-5, over
    ctx.set_tuning(**DEFAULT)


@pytest.mark.parametrize("precision", [snk.SNK_MIXED, snk.SNK_FP32])
def test_autotune_picks_valid_shapes_and_leaves_the_training_state(ctx, precision):
    case = make_case("window2x2_full", n_rays=2048, crop=48, table_scale=0.3)
    crops = [dev(t.astype(np.float32)) for t in case.targets]
    ctx.set_views(case.cams, crops)
    w = case.w
    tr = Trainer(ctx, model_from_workload(w, precision), snk.window_struct(w.window()),
                 snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 5, 0), case.params)
    before = [x.clone() for x in (tr.params, tr.grads, tr.m, tr.v, tr.steps, tr.state)]
    t = tr.autotune(dev(case.pix.view(np.int32)))
    torch.cuda.synchronize()
    assert t["tuned"] == 1
    assert t["tc_fwd_ctas"] in (1, 2, 3) and t["tc_fwd_levels"] in (1, 2) and t["fp32_ctas"] in (1, 2)
    assert t["tc_fwd_split"] in (0, 1) and t["tc_bwd_saved"] in (0, 1)
    assert t["composite_threads"] in (64, 128, 256, 512) and t["sampler_threads"] in (128, 256, 512)
    assert ctx.tuning() == t
    for a, b in zip(before, (tr.params, tr.grads, tr.m, tr.v, tr.steps, tr.state)):
        assert torch.equal(a, b)
    # a step with the tuned shapes still trains
    tr.train_step(dev(case.pix.view(np.int32)))
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    ctx.set_tuning(**DEFAULT)
    assert ctx.tuning()["tuned"] == 0


def test_out_of_range_tuning_is_rejected(ctx):
    for key, val in [("tc_fwd_ctas", 4), ("tc_fwd_levels", 4), ("tc_bwd_saved", 2), ("tc_fwd_split", 2),
                     ("composite_threads", 96 + 1),
                     ("sampler_threads", 1024), ("fp32_ctas", 0)]:
        with pytest.raises(RuntimeError):
            ctx.set_tuning(**dict(DEFAULT, **{key: val}))
    with pytest.raises(KeyError):  # a misspelled field is not silently ignored
        ctx.set_tuning(tc_fwd_splits=0)
    assert ctx.tuning()["tc_fwd_ctas"] == DEFAULT["tc_fwd_ctas"]
