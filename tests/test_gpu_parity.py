"""CUDA library vs FP64 oracle, element by element, through the C ABI.

Bit-exact: rays (binary32 rounding of the binary64 camera), acceptance,
segment tiles and bounds, samples per segment, sample positions, hash entry
indices.  Floats: rendered RGB and depth within rel 1e-5 of the oracle (with
a floor of rel x max|value| for near-zero entries); gradients within 5e-4
norm-wise per tensor (binary32 accumulation and atomic order)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from oracle import camera, hashgrid, mlp, render, sampler, step as OS
import synth
from gpu_util import (GRAD_REL_FP32, RGB_REL_FP32, close, gpu_to_ray_major, make_case, normwise)

pytestmark = pytest.mark.gpu
U32 = np.uint32
# |computed - exact| <= BOUND_U * (the same computation on absolute values): 500 unit roundoffs of
# binary32 covers 64-term dot products chained through 6 layers plus the per-thread sums over samples
BOUND_U = 500 * 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.view(dtype)
    return t.cuda()


def run_sampling(ctx, case, seed=7, iteration=3, render=0, cap=None):
    w = case.w
    B = len(case.pix)
    win = case.w.window()
    ws = snk.window_struct(win)
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, render, seed, iteration)
    ctx.set_views(case.cams)
    nseg = 1 + (w.nx == 2) + (w.ny == 2)
    if cap is None:
        cap = B * nseg * w.K_max + 4 * 128
    f32, i32, u8 = torch.float32, torch.int32, torch.uint8
    g = {
        "pix": dev(case.pix.view(np.int32)),
        "ray_od": torch.zeros(6 * B, dtype=f32, device="cuda"),
        "ray_ok": torch.zeros(B, dtype=u8, device="cuda"),
        "seg_slot": torch.zeros(3 * B, dtype=u8, device="cuda"),
        "seg_t": torch.zeros(6 * B, dtype=f32, device="cuda"),
        "seg_n": torch.zeros(3 * B, dtype=i32, device="cuda"),
        "seg_off": torch.zeros(3 * B, dtype=i32, device="cuda"),
        "smp_t": torch.zeros(max(cap, 1), dtype=f32, device="cuda"),
        "smp_dt": torch.zeros(max(cap, 1), dtype=f32, device="cuda"),
        "smp_xyz": torch.zeros(3 * max(cap, 1), dtype=f32, device="cuda"),
        "state": torch.zeros(snk.STATE_WORDS, dtype=i32, device="cuda"),
    }
    ctx.call("snk_sample_segments", ctypes.byref(ws), snk.ptr(g["pix"]), B, ctypes.byref(sp), snk.ptr(g["ray_od"]),
             snk.ptr(g["ray_ok"]), snk.ptr(g["seg_slot"]), snk.ptr(g["seg_t"]), snk.ptr(g["seg_n"]),
             snk.ptr(g["seg_off"]), snk.ptr(g["smp_t"]), snk.ptr(g["smp_dt"]), snk.ptr(g["smp_xyz"]), cap,
             snk.ptr(g["state"]), None)
    torch.cuda.synchronize()
    h = {k: v.cpu().numpy() for k, v in g.items()}
    h["cap"] = cap
    h["dev"] = g
    st = h["state"]
    h["slot_base"] = st[7:12].view(U32)
    h["slot_count"] = st[12:16].view(U32)
    h["n_accepted"] = int(st[2:3].view(U32)[0])
    h["n_samples"] = int(st[3:4].view(U32)[0])
    h["status"] = int(st[4:5].view(U32)[0])
    return h


def oracle_sampling(case, seed=7, iteration=3, render=False):
    w = case.w
    win = w.window()
    o, d = camera.rays(case.cams, case.pix, win.origin, win.origin[2], win.origin[2] + win.tile_size[2])
    wf = sampler.window_f32(win)
    seg = sampler.segments(o, d, wf, w.K_ray, w.K_min, w.K_max)
    smp = sampler.stratified(o, d, seg, wf, seed, iteration, render=render)
    return o, d, seg, smp


SAMPLING_CASES = [("tiny_tile", 96), ("tiny_window", 160), ("tile256_fp32", 1024), ("tile512_full", 2500),
                  ("window2x2_full", 2500)]


@pytest.mark.parametrize("name,n_rays", SAMPLING_CASES)
@pytest.mark.parametrize("render", [0, 1])
def test_rays_segments_samples_bit_exact(ctx, name, n_rays, render):
    case = make_case(name, n_rays=n_rays, with_targets=False)
    g = run_sampling(ctx, case, render=render)
    o, d, seg, smp = oracle_sampling(case, render=bool(render))
    B = n_rays
    od = g["ray_od"].reshape(6, B)
    assert np.array_equal(od[:3].T, o) and np.array_equal(od[3:].T, d), "rays differ from the oracle"
    assert np.array_equal(g["ray_ok"], seg.ray_ok)
    assert g["status"] == 0
    seg_slot = g["seg_slot"].reshape(B, 3).astype(np.int64)
    seg_t = g["seg_t"].reshape(B, 3, 2)
    seg_n = g["seg_n"].reshape(B, 3)
    seg_off = g["seg_off"].reshape(B, 3)
    assert np.array_equal(seg_slot, seg.slot)
    assert np.array_equal(seg_t[..., 0], seg.t0) and np.array_equal(seg_t[..., 1], seg.t1)
    assert np.array_equal(seg_n, seg.K)
    assert g["n_accepted"] == int(seg.ray_ok.sum())
    assert g["n_samples"] == int(seg.ray_off[-1])
    for k in range(case.w.n_slots):
        assert g["slot_count"][k] == int(seg.K[seg.slot == k].sum())
        assert g["slot_base"][k] % 128 == 0
    idx = gpu_to_ray_major(seg_n, seg_off, seg.ray_off)
    assert np.array_equal(g["smp_t"][idx], smp.t)
    assert np.array_equal(g["smp_dt"][idx], smp.dt)
    assert np.array_equal(g["smp_xyz"].reshape(-1, 3)[idx], smp.xyz)
    # every sample index is used once and lies inside its slot's range
    assert len(np.unique(idx)) == len(idx)
    for k in range(case.w.n_slots):
        m = smp.slot == k
        assert np.all((idx[m] >= g["slot_base"][k]) & (idx[m] < g["slot_base"][k] + g["slot_count"][k]))


def _model_and_params(case, precision=snk.SNK_FP32):
    model = model_from_workload(case.w, precision)
    lay = snk.layout(model)
    p = dev(case.params)
    grads = torch.zeros(lay.n_params, dtype=torch.float32, device="cuda")
    ps = snk.SnkParams(snk.ptr(p), None, snk.ptr(grads), None, None, None)
    return model, lay, p, grads, ps


@pytest.mark.parametrize("name,n_rays", [("tiny_window", 160), ("tile256_fp32", 512), ("tile512_full", 600)])
def test_encode_indices_bit_exact_and_features(ctx, name, n_rays):
    case = make_case(name, n_rays=n_rays, with_targets=False, table_scale=0.5)
    g = run_sampling(ctx, case)
    o, d, seg, smp = oracle_sampling(case)
    model, lay, p, grads, ps = _model_and_params(case)
    cap = g["cap"]
    L, F = case.w.L, case.w.F
    feat = torch.zeros(cap * L * F, dtype=torch.float32, device="cuda")
    idx_out = torch.zeros(cap * L * 8, dtype=torch.int32, device="cuda")
    ctx.call("snk_encode", ctypes.byref(model), ctypes.byref(ps), snk.ptr(g["dev"]["smp_xyz"]),
             snk.ptr(g["dev"]["state"]), cap, snk.ptr(feat), snk.ptr(idx_out), None)
    torch.cuda.synchronize()
    idx = gpu_to_ray_major(g["seg_n"].reshape(-1, 3), g["seg_off"].reshape(-1, 3), seg.ray_off)
    gi = idx_out.cpu().numpy().reshape(cap, L, 8)[idx]
    gf = feat.cpu().numpy().reshape(cap, L * F)[idx]
    cfg = case.cfg
    tiles, _ = OS.unflatten(cfg, case.params.astype(np.float64))
    glay = cfg.grid()
    for k in range(case.w.n_slots):
        m = smp.slot == k
        if not m.any():
            continue
        for l in range(L):
            ci, _ = hashgrid.corners(smp.xyz[m], glay, l)
            assert np.array_equal(gi[m, l, :].astype(np.int64), ci), "hash indices differ (slot %d level %d)" % (k, l)
        ref = hashgrid.encode(smp.xyz[m], tiles[k][0], glay)
        ok, err = close(gf[m], ref, 1e-5)
        assert ok, err


@pytest.mark.parametrize("name,n_rays", [("tiny_window", 160), ("tile256_fp32", 512), ("tile512_full", 600)])
def test_mlp_forward_and_backward(ctx, name, n_rays):
    case = make_case(name, n_rays=n_rays, with_targets=False, table_scale=0.5)
    g = run_sampling(ctx, case)
    o, d, seg, smp = oracle_sampling(case)
    model, lay, p, grads, ps = _model_and_params(case)
    cap = g["cap"]
    IN = case.w.L * case.w.F
    rng = np.random.default_rng(1)
    feat_h = rng.normal(0, 0.5, (cap, IN)).astype(np.float32)
    feat = dev(feat_h)
    out = torch.zeros(cap * 4, dtype=torch.float32, device="cuda")
    ctx.call("snk_mlp", ctypes.byref(model), ctypes.byref(ps), snk.ptr(feat), snk.ptr(g["dev"]["state"]), cap,
             snk.ptr(out), None)
    dout_h = rng.normal(0, 1.0, (cap, 4)).astype(np.float32)
    dout = dev(dout_h)
    dfeat = torch.zeros(cap * IN, dtype=torch.float32, device="cuda")
    ctx.call("snk_mlp_backward", ctypes.byref(model), ctypes.byref(ps), snk.ptr(feat), snk.ptr(g["dev"]["state"]),
             cap, snk.ptr(dout), snk.ptr(dfeat), None)
    torch.cuda.synchronize()
    idx = gpu_to_ray_major(g["seg_n"].reshape(-1, 3), g["seg_off"].reshape(-1, 3), seg.ray_off)
    go = out.cpu().numpy().reshape(cap, 4)[idx]
    gdf = dfeat.cpu().numpy().reshape(cap, IN)[idx]
    gg = grads.cpu().numpy().astype(np.float64)
    cfg = case.cfg
    flat = case.params.astype(np.float64)
    tiles, cols = OS.unflatten(cfg, flat)
    ref_grad = np.zeros_like(flat)
    gt_, gc_ = OS.unflatten(cfg, ref_grad)
    abs_grad = np.zeros_like(flat)
    at_, ac_ = OS.unflatten(cfg, abs_grad)
    x = feat_h[idx].astype(np.float64)
    dd = dout_h[idx].astype(np.float64)
    # A ReLU mask is a decision taken by a float: where a pre-activation lies within binary32
    # rounding of zero (|z| < 1e-5 sum|w x|) the two precisions may decide differently.  Such
    # samples get a zero upstream gradient on both sides, so their masks cannot matter.
    amb = np.zeros(cap, bool)
    amb_r = np.zeros(len(idx), bool)
    for k in range(case.w.n_slots):
        m = smp.slot == k
        if not m.any():
            continue
        col = (cols[0] if cfg.shared_colour else cols[k]) if cfg.colour else None
        _, _, acts = mlp.forward(x[m], tiles[k][1], col)
        gp = acts["geo_pre"]
        hidden = [(acts["x0"], tiles[k][1][0], gp[0]), (np.maximum(gp[0], 0), tiles[k][1][1], gp[1])]
        if col is not None:
            cp = acts["col_pre"]
            hidden += [(acts["g"], col[0], cp[0]), (np.maximum(cp[0], 0), col[1], cp[1])]
        bad = np.zeros(int(m.sum()), bool)
        for h, Wm, z in hidden:            # the ReLU layers; output layers have no mask
            bad |= np.any(np.abs(z) < 1e-5 * (np.abs(h) @ np.abs(Wm).T), axis=1)
        amb_r[np.flatnonzero(m)[bad]] = True
    amb[idx[amb_r]] = True
    dout_h[amb] = 0.0
    dd[amb_r] = 0.0
    dout.copy_(torch.from_numpy(dout_h))
    grads.zero_()
    ctx.call("snk_mlp_backward", ctypes.byref(model), ctypes.byref(ps), snk.ptr(feat), snk.ptr(g["dev"]["state"]),
             cap, snk.ptr(dout), snk.ptr(dfeat), None)
    torch.cuda.synchronize()
    gdf = dfeat.cpu().numpy().reshape(cap, IN)[idx]
    gg = grads.cpu().numpy().astype(np.float64)
    for k in range(case.w.n_slots):
        m = smp.slot == k
        if not m.any():
            continue
        col = (cols[0] if cfg.shared_colour else cols[k]) if cfg.colour else None
        s_, c_, acts = mlp.forward(x[m], tiles[k][1], col)
        ok, err = close(go[m, 0], s_, RGB_REL_FP32)
        assert ok, ("sigma", err)
        ok, err = close(go[m, 1:], c_, RGB_REL_FP32)
        assert ok, ("rgb", err)
        dgeo, dcol, dx = mlp.backward(dd[m, 0], dd[m, 1:], tiles[k][1], col, acts)
        # running-error bound: the same backward on absolute values (|W|, |inputs|, |upstream|, same
        # ReLU masks) bounds sum |terms| of every accumulated quantity
        acts_abs = dict(acts)
        acts_abs["x0"] = np.abs(acts["x0"])
        acts_abs["g"] = np.abs(acts["g"])
        if "col_in" in acts:  # the colour layer's input, [g] or [g | SH(d)]
            acts_abs["col_in"] = np.abs(acts["col_in"])
        ageo, acol, adx = mlp.backward(np.abs(dd[m, 0]), np.abs(dd[m, 1:]), [np.abs(W) for W in tiles[k][1]],
                                       [np.abs(V) for V in col] if col is not None else None, acts_abs)
        for q in range(3):
            gt_[k][1][q] += dgeo[q]
            at_[k][1][q] += ageo[q]
            if cfg.colour:
                (gc_[0] if cfg.shared_colour else gc_[k])[q] += dcol[q]
                (ac_[0] if cfg.shared_colour else ac_[k])[q] += acol[q]
        assert np.all(np.abs(gdf[m] - dx) <= BOUND_U * adx + 1e-30)
    gtiles, gcols = OS.unflatten(cfg, gg)
    for k in range(case.w.n_slots):
        for q in range(3):
            assert np.all(np.abs(gtiles[k][1][q] - gt_[k][1][q]) <= BOUND_U * at_[k][1][q] + 1e-30), ("geo", k, q)
    for c in range(len(gcols)):
        for q in range(3):
            assert np.all(np.abs(gcols[c][q] - gc_[c][q]) <= BOUND_U * ac_[c][q] + 1e-30), ("colour", c, q)
    # tables untouched by the MLP-only backward
    assert np.all(gg[:lay.grid_params] == 0)


@pytest.mark.parametrize("name,n_rays", [("tiny_window", 160), ("tile512_full", 600), ("window2x2_full", 800)])
def test_composite_forward_and_backward(ctx, name, n_rays):
    case = make_case(name, n_rays=n_rays, with_targets=False)
    g = run_sampling(ctx, case)
    o, d, seg, smp = oracle_sampling(case)
    cap = g["cap"]
    B = n_rays
    rng = np.random.default_rng(2)
    sr_h = np.zeros((cap, 4), np.float32)
    sr_h[:, 0] = rng.gamma(1.0, 0.05, cap)
    sr_h[:, 1:] = rng.uniform(0, 1, (cap, 3))
    sr = dev(sr_h)
    out = torch.zeros(B * 5, dtype=torch.float32, device="cuda")
    tfin = torch.zeros(B, dtype=torch.float32, device="cuda")
    D = g["dev"]
    ctx.call("snk_composite", snk.ptr(sr), snk.ptr(D["smp_t"]), snk.ptr(D["smp_dt"]), snk.ptr(D["seg_n"]),
             snk.ptr(D["seg_off"]), B, snk.ptr(out), snk.ptr(tfin), None)
    g_rgb_h = rng.normal(0, 1, (B, 3)).astype(np.float32)
    g_rgb = dev(g_rgb_h)
    dsr = torch.zeros(cap * 4, dtype=torch.float32, device="cuda")
    ctx.call("snk_composite_backward", snk.ptr(sr), snk.ptr(D["smp_t"]), snk.ptr(D["smp_dt"]), snk.ptr(D["seg_n"]),
             snk.ptr(D["seg_off"]), B, snk.ptr(g_rgb), snk.ptr(dsr), None)
    torch.cuda.synchronize()
    idx = gpu_to_ray_major(g["seg_n"].reshape(-1, 3), g["seg_off"].reshape(-1, 3), seg.ray_off)
    s = sr_h[idx].astype(np.float64)
    rgb, depth, op, tf, _ = render.composite(s[:, 0], s[:, 1:], smp.t.astype(np.float64), smp.dt.astype(np.float64),
                                             seg.ray_off)
    go = out.cpu().numpy().reshape(B, 5)
    for name_, a, b in [("rgb", go[:, :3], rgb), ("depth", go[:, 3], depth), ("opacity", go[:, 4], op),
                        ("T_final", tfin.cpu().numpy(), tf)]:
        ok, err = close(a, b, RGB_REL_FP32)
        assert ok, (name_, err)
    dsig, drgb = render.composite_backward(g_rgb_h.astype(np.float64), s[:, 0], s[:, 1:],
                                           smp.t.astype(np.float64), smp.dt.astype(np.float64), seg.ray_off)
    gd = dsr.cpu().numpy().reshape(cap, 4)[idx]
    assert normwise(gd[:, 0], dsig) < GRAD_REL_FP32
    assert normwise(gd[:, 1:], drgb) < GRAD_REL_FP32


def test_composite_long_rays_and_segment_edges(ctx):
    """Synthetic segment counts around the compositing kernel's shared-memory limit for a ray's
    weights (16 chunks of 32 samples): rays of exactly 512 samples keep them on chip, longer
    ones (513, 700 and 900 samples) park them in the gradient buffer; also segments of one
    sample, segments that end a chunk early, and an empty ray.  Forward and backward against
    the oracle's compositing."""
    counts = np.array([[512, 0, 0], [513, 0, 0], [400, 200, 100], [300, 300, 300], [31, 1, 0], [1, 1, 1],
                       [0, 0, 0], [33, 64, 65], [0, 17, 0], [256, 0, 256]], np.int64)
    B = len(counts)
    rng = np.random.default_rng(11)
    n = int(counts.sum())
    seg_off = np.zeros((B, 3), np.int64)
    ray_off = np.zeros(B + 1, np.int64)
    t = np.zeros(n, np.float32)
    dt = np.zeros(n, np.float32)
    p = 0
    for r in range(B):
        ray_off[r] = p
        tt = 0.0
        for sgm in range(3):
            seg_off[r, sgm] = p
            for _ in range(counts[r, sgm]):
                d = rng.uniform(0.01, 0.2)
                t[p], dt[p] = tt + 0.5 * d, d
                tt += d
                p += 1
    ray_off[B] = p
    sr_h = np.zeros((n, 4), np.float32)
    sr_h[:, 0] = rng.gamma(1.0, 0.02, n)
    sr_h[:, 1:] = rng.uniform(0, 1, (n, 3))
    sr, td, dtd = dev(sr_h), dev(t), dev(dt)
    sn, so = dev(counts.astype(np.int32)), dev(seg_off.astype(np.int32))
    out = torch.zeros(B * 5, dtype=torch.float32, device="cuda")
    tfin = torch.zeros(B, dtype=torch.float32, device="cuda")
    ctx.call("snk_composite", snk.ptr(sr), snk.ptr(td), snk.ptr(dtd), snk.ptr(sn), snk.ptr(so), B, snk.ptr(out),
             snk.ptr(tfin), None)
    g_rgb_h = rng.normal(0, 1, (B, 3)).astype(np.float32)
    dsr = torch.zeros(n * 4, dtype=torch.float32, device="cuda")
    ctx.call("snk_composite_backward", snk.ptr(sr), snk.ptr(td), snk.ptr(dtd), snk.ptr(sn), snk.ptr(so), B,
             snk.ptr(dev(g_rgb_h)), snk.ptr(dsr), None)
    torch.cuda.synchronize()
    s64 = sr_h.astype(np.float64)
    rgb, depth, op, tf, _ = render.composite(s64[:, 0], s64[:, 1:], t.astype(np.float64), dt.astype(np.float64),
                                             ray_off)
    go = out.cpu().numpy().reshape(B, 5)
    for name_, a, b in [("rgb", go[:, :3], rgb), ("depth", go[:, 3], depth), ("opacity", go[:, 4], op),
                        ("T_final", tfin.cpu().numpy(), tf)]:
        ok, err = close(a, b, RGB_REL_FP32)
        assert ok, (name_, err)
    dsig, drgb = render.composite_backward(g_rgb_h.astype(np.float64), s64[:, 0], s64[:, 1:], t.astype(np.float64),
                                           dt.astype(np.float64), ray_off)
    gd = dsr.cpu().numpy().reshape(n, 4)
    for r in range(B):  # per ray, so that a wrong chunk on one path cannot hide in the norm
        a, b = ray_off[r], ray_off[r + 1]
        if b > a:
            assert normwise(gd[a:b, 0], dsig[a:b]) < GRAD_REL_FP32, r
            assert normwise(gd[a:b, 1:], drgb[a:b]) < GRAD_REL_FP32, r


def _trainer(ctx, case, precision=snk.SNK_FP32, seed=5):
    w = case.w
    crops = [dev(t.astype(np.float32)) for t in case.targets]
    ctx.set_views(case.cams, crops)
    model = model_from_workload(w, precision)
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, seed, 0)
    tr = Trainer(ctx, model, snk.window_struct(w.window()), sp, case.params)
    tr._crops = crops
    return tr


@pytest.mark.parametrize("name,n_rays,crop", [("tiny_tile", 96, None), ("tiny_window", 160, None),
                                              ("tile256_fp32", 1024, None), ("tile512_full", 512, 48)])
def test_train_step_fp32_matches_oracle(ctx, name, n_rays, crop):
    case = make_case(name, n_rays=n_rays, crop=crop, table_scale=0.3)
    tr = _trainer(ctx, case)
    B = n_rays
    out = torch.zeros(B * 5, dtype=torch.float32, device="cuda")
    pix = dev(case.pix.view(np.int32))
    tr.train_step(pix, out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    st = tr.read_state()
    n = len(case.params)
    flat = case.params.astype(np.float64)
    ref = OS.train_step(case.cfg, flat, np.zeros(n), np.zeros(n), [0] * case.cfg.n_optimisers(), case.cams,
                        case.w.window(), case.pix, case.targets, 5, 0)
    assert st["iteration"] == 1
    assert st["n_accepted"] == int(ref.seg.ray_ok.sum())
    assert st["n_samples"] == int(ref.seg.ray_off[-1])
    ok, err = close([st["loss"]], [ref.loss], RGB_REL_FP32)
    assert ok, ("loss", st["loss"], ref.loss)
    go = out.cpu().numpy().reshape(B, 5)
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a, b, RGB_REL_FP32)
        assert ok, (nm, err)
    # first Adam step: m = (1 - beta1) (g + decay)  -> compare the gradients through m
    m = tr.m.cpu().numpy().astype(np.float64)
    ref_m = ref.m
    for gi, (a, b, mlp_a) in enumerate(OS.group_ranges(case.cfg)):
        if mlp_a > a:
            assert normwise(m[a:mlp_a], ref_m[a:mlp_a]) < GRAD_REL_FP32, ("table", gi)
        assert normwise(m[mlp_a:b], ref_m[mlp_a:b]) < GRAD_REL_FP32, ("mlp", gi)
        # parameters: where the gradient is clearly non-zero the first step moves by lr sign(g)
        pg = tr.params.cpu().numpy().astype(np.float64)[a:b]
        rg = np.abs(ref.grad[a:b])
        sure = rg > 1e-3 * max(rg.max(), 1e-30)
        assert np.allclose(pg[sure], ref.params[a:b][sure], rtol=0, atol=1e-6)
    assert np.all(tr.steps.cpu().numpy() == 1)
    assert np.all(tr.grads.cpu().numpy() == 0), "the step must leave the gradient accumulator zeroed"


@pytest.mark.parametrize("name,n_rays,crop", [("tiny_window", 160, None), ("tile512_full", 400, None),
                                              ("window2x2_full", 600, None)])
def test_render_fp32_matches_oracle(ctx, name, n_rays, crop):
    case = make_case(name, n_rays=n_rays, crop=crop, table_scale=0.3, with_targets=False)
    case.targets = None
    ctx.set_views(case.cams)
    model = model_from_workload(case.w, snk.SNK_FP32)
    sp = snk.sampler_struct(case.w.K_ray, case.w.K_min, case.w.K_max, 1, 0, 0)
    tr = Trainer(ctx, model, snk.window_struct(case.w.window()), sp, case.params)
    out = torch.zeros(n_rays * 5, dtype=torch.float32, device="cuda")
    tr.render(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    ref = OS.render_rays(case.cfg, case.params.astype(np.float64), case.cams, case.w.window(), case.pix)
    go = out.cpu().numpy().reshape(n_rays, 5)
    for nm, a, b in [("rgb", go[:, :3], ref.rgb), ("depth", go[:, 3], ref.depth), ("opacity", go[:, 4], ref.opacity)]:
        ok, err = close(a, b, RGB_REL_FP32)
        assert ok, (nm, err)


def test_rays_missing_the_box_give_empty_batches(ctx):
    """Pixels whose rays miss the scene box: nothing accepted, no samples, zero
    loss, rendering black, no device check."""
    case = make_case("tiny_tile", n_rays=64, table_scale=0.3)
    # far outside the 48-px images: the localised points are kilometres away
    case.pix = synth.pack_pixel(np.zeros(64, int), np.full(64, 4000), np.arange(64) + 3000)
    for c in case.cams:
        c.crop = (3990, 2990, 100, 100)
    case.targets = [np.zeros((100, 100, 3), np.float32) for _ in case.cams]
    tr = _trainer(ctx, case)
    out = torch.full((64 * 5,), 7.0, dtype=torch.float32, device="cuda")
    tr.train_step(dev(case.pix.view(np.int32)), out)
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    st = tr.read_state()
    assert st["n_accepted"] == 0 and st["n_samples"] == 0 and st["loss"] == 0.0
    assert np.all(out.cpu().numpy() == 0)


def test_sample_capacity_overflow_is_reported_not_written(ctx):
    case = make_case("tiny_window", n_rays=160, with_targets=False)
    g = run_sampling(ctx, case, cap=100)
    assert g["status"] & snk.STATUS_CHECK
    assert g["n_samples"] == 0 and np.all(g["slot_count"] == 0)
    assert np.all(g["smp_t"] == 0)
    assert ctx.sync_status(g["dev"]["state"]) == snk.SNK_ERR_DEVICE_CHECK


def test_invalid_view_index_sets_the_device_check(ctx):
    case = make_case("tiny_tile", n_rays=32, with_targets=False)
    case.pix = case.pix.copy()
    case.pix[5] = synth.pack_pixel(200, 3, 3)
    g = run_sampling(ctx, case)
    assert g["ray_ok"][5] == 0 and g["status"] & snk.STATUS_CHECK
