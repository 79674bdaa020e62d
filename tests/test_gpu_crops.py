"""Crops, ray pool and batch draw on the device against the oracle.

Crop rectangles: exact, except a bound whose corner projection lies within
1e-6 pixel of an integer (the floor or ceiling may go either way between two
binary64 iterations), which may differ by one.  The pool is built from the
oracle's own rectangles and must equal the oracle's pool entry by entry (the
acceptance is bit-exact), the draw likewise; and a training step on a drawn
batch accepts every ray."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import crops as C
from synth import workloads as W

pytestmark = pytest.mark.gpu
AMBIGUOUS = 1e-6


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def _near_int(x):
    return abs(x - round(x)) < AMBIGUOUS


def _bounds_ok(got, want, proj, margin):
    """got/want (r0, c0, h, w); a bound may differ by 1 if its extreme projection is near an integer."""
    g = (got[0], got[1], got[0] + got[2], got[1] + got[3])
    w = (want[0], want[1], want[0] + want[2], want[1] + want[3])
    ext = (proj[:, 0].min(), proj[:, 1].min(), proj[:, 0].max(), proj[:, 1].max())
    for a, b, e in zip(g, w, ext):
        if a != b and not (abs(a - b) == 1 and _near_int(e)):
            return False
    return True


CASES = [("tiny_sweep", (0, 0), 2), ("tiny_sweep", (1, 1), 4), ("window2x2_full", (0, 0), 64),
         ("sweep_grid8", (3, 5), 64), ("tile256_fp32", (0, 0), 0)]


@pytest.mark.parametrize("name,pos,margin", CASES)
def test_crops_match_the_oracle(ctx, name, pos, margin):
    w = W.get(name)
    cams = W.cameras(w)
    ctx.set_views(cams)
    win = w.window(pos)
    nv = len(cams)
    tr = torch.zeros(nv * 16, dtype=torch.int32, device="cuda")
    vr = torch.zeros(nv * 4, dtype=torch.int32, device="cuda")
    ctx.call("snk_build_crops", ctypes.byref(snk.window_struct(win)), margin, snk.ptr(tr), snk.ptr(vr), None)
    torch.cuda.synchronize()
    tiles, views, proj = C.crops(cams, win, margin)
    gt = tr.cpu().numpy().reshape(nv, 4, 4)
    gv = vr.cpu().numpy().reshape(nv, 4)
    n_tiles = w.nx * w.ny
    for v in range(nv):
        for k in range(n_tiles):
            assert _bounds_ok(tuple(gt[v, k]), tiles[v][k], proj[v][k], margin), (v, k, gt[v, k], tiles[v][k])
        assert np.all(gt[v, n_tiles:] == 0)
        allp = np.concatenate(proj[v])
        assert _bounds_ok(tuple(gv[v]), views[v], allp, margin) or tuple(gv[v]) == tuple(views[v]), (v, gv[v], views[v])


@pytest.mark.parametrize("name,pos,margin", CASES[:3])
def test_pool_and_draw_match_the_oracle(ctx, name, pos, margin):
    w = W.get(name)
    cams = W.cameras(w)
    ctx.set_views(cams)
    win = w.window(pos)
    _, views, _ = C.crops(cams, win, margin)
    want = C.ray_pool(cams, win, views)
    vr = torch.tensor(np.array(views, np.int32).ravel(), device="cuda")
    cap = max(len(want), 1)
    pool = torch.zeros(cap, dtype=torch.int32, device="cuda")
    n = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.call("snk_ray_pool", ctypes.byref(snk.window_struct(win)), snk.ptr(vr), snk.ptr(pool), cap, snk.ptr(n), None)
    torch.cuda.synchronize()
    nn = n.cpu().numpy().view(np.uint32)
    assert nn[0] == len(want) and nn[1] == len(want)
    assert np.array_equal(pool.cpu().numpy().view(np.uint32)[:len(want)], want)
    # a pool too small for the crops: filled to cap, the full count reported
    if len(want) > 10:
        small = torch.zeros(10, dtype=torch.int32, device="cuda")
        ctx.call("snk_ray_pool", ctypes.byref(snk.window_struct(win)), snk.ptr(vr), snk.ptr(small), 10, snk.ptr(n),
                 None)
        torch.cuda.synchronize()
        nn = n.cpu().numpy().view(np.uint32)
        assert nn[0] == 10 and nn[1] == len(want)
        assert np.array_equal(small.cpu().numpy().view(np.uint32), want[:10])
    B = 5000
    pix = torch.zeros(B, dtype=torch.int32, device="cuda")
    n_dev = torch.tensor(np.array([len(want), len(want)], np.uint32).view(np.int32), device="cuda")
    ctx.call("snk_draw_batch", snk.ptr(pool), snk.ptr(n_dev), B, 11, 3, snk.ptr(pix), None)
    torch.cuda.synchronize()
    assert np.array_equal(pix.cpu().numpy().view(np.uint32), C.draw(want, B, 11, 3))


def test_a_step_on_a_drawn_batch_accepts_every_ray(ctx):
    w = W.get("window2x2_full")
    cams = W.cameras(w)
    win = w.window()
    crops = [torch.zeros(c.crop[2] * c.crop[3] * 3, dtype=torch.float32, device="cuda") for c in cams]
    ctx.set_views(cams, crops)
    nv = len(cams)
    tr_ = torch.zeros(nv * 16, dtype=torch.int32, device="cuda")
    vr = torch.zeros(nv * 4, dtype=torch.int32, device="cuda")
    ws = snk.window_struct(win)
    ctx.call("snk_build_crops", ctypes.byref(ws), 64, snk.ptr(tr_), snk.ptr(vr), None)
    cap = 1 << 26
    pool = torch.zeros(cap, dtype=torch.int32, device="cuda")
    n = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.call("snk_ray_pool", ctypes.byref(ws), snk.ptr(vr), snk.ptr(pool), cap, snk.ptr(n), None)
    B = 65536
    pix = torch.zeros(B, dtype=torch.int32, device="cuda")
    ctx.call("snk_draw_batch", snk.ptr(pool), snk.ptr(n), B, 1, 0, snk.ptr(pix), None)
    model = model_from_workload(w)
    lay = snk.layout(model)
    geo = [(64, w.L * w.F), (64, 64), (w.geo_out, 64)]
    col = [(64, w.geo_out), (64, 64), (3, 64)]
    params = W.init_params(lay.grid_params, geo, col, w.n_slots, 1, 0)
    t = Trainer(ctx, model, ws, snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 1, 0), params)
    t.train_step(pix)
    assert ctx.sync_status(t.state) == snk.SNK_OK
    assert t.read_state()["n_accepted"] == B
