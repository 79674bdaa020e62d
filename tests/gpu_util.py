"""Helpers shared by the GPU parity tests: build the same seeded case for the
CUDA library and for the FP64 oracle, and map the library's slot-major sample
arrays onto the oracle's ray-major order."""
import dataclasses

import numpy as np

import synth
from synth import workloads as W
from oracle import step as OS, targets as OT

RGB_REL_FP32 = 1e-5      # rendered RGB and depth, binary32 path
GRAD_REL_FP32 = 5e-4     # gradients (norm-wise per tensor), binary32 path: 6 chained 64-term
#                          binary32 dot products, u = 6e-8, ~sqrt(64) random-sign cancellation each: ~1.8e-4
RGB_REL_MIXED = 2e-3
GRAD_REL_MIXED = 5e-3


def close(a, b, rel):
    """Elementwise |a - b| <= rel |b| + rel max|b| (floor for near-zero entries)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    floor = rel * (np.max(np.abs(b)) if b.size else 0.0)
    err = np.abs(a - b) - (rel * np.abs(b) + floor)
    return bool(np.all(err <= 0)), float(np.max(np.abs(a - b)) if a.size else 0.0)


def normwise(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def small_crops(cams, size, seed=0):
    """Shrink every view's crop to a size x size square near the image centre
    (keeps oracle target rendering cheap for the full-size cameras)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in cams:
        h = min(size, c.height)
        w = min(size, c.width)
        r0 = int(rng.integers(max(0, c.height // 2 - 2 * h), max(1, c.height // 2 + h)))
        c0 = int(rng.integers(max(0, c.width // 2 - 2 * w), max(1, c.width // 2 + w)))
        r0 = min(r0, c.height - h)
        c0 = min(c0, c.width - w)
        out.append(dataclasses.replace(c, crop=(r0, c0, h, w)))
    return out


def model_config(w, hidden=64):
    return OS.ModelConfig(L=w.L, F=w.F, log2_T=w.log2_T, n_min=w.n_min, n_max=w.n_max, hidden=hidden,
                          geo_out=w.geo_out, colour=w.colour, shared_colour=w.shared_colour, n_slots=w.n_slots,
                          K_ray=w.K_ray, K_min=w.K_min, K_max=w.K_max, first_layer=w.first_layer,
                          view_dirs=w.view_dirs)


@dataclasses.dataclass
class Case:
    w: object
    cams: list
    targets: list
    cfg: object
    params: np.ndarray
    pix: np.ndarray


def make_case(name, n_rays=None, crop=None, seed=0, table_scale=None, with_targets=True, **over):
    w = W.get(name, **over) if over else W.get(name)
    if n_rays is not None:
        w = dataclasses.replace(w, n_rays=n_rays)
    cams = W.cameras(w)
    if crop is not None:
        cams = small_crops(cams, crop, seed)
    targets = OT.render_targets(W.scene(w), cams) if with_targets else None
    cfg = model_config(w)
    lay = cfg.grid()
    params = W.init_params(lay.n_params, cfg.geo_shapes(), cfg.col_shapes(), cfg.n_slots, cfg.n_colour_blocks(),
                           seed)
    if table_scale is not None:
        rng = np.random.default_rng(seed + 5)
        for a, b, mlp_a in OS.group_ranges(cfg)[:cfg.n_slots]:
            params[a:mlp_a] = rng.uniform(-table_scale, table_scale, mlp_a - a).astype(np.float32)
    # with shrunken crops every pixel is drawn inside its view's crop
    pix = synth.random_pixels(seed + 3, w.n_rays, cams) if crop is not None else W.batch(w, cams, seed + 3)
    return Case(w, cams, targets, cfg, params, pix)


def gpu_to_ray_major(seg_n, seg_off, ray_off_oracle):
    """Index into the slot-major arrays for every oracle (ray-major) sample."""
    B = seg_n.shape[0]
    idx = np.zeros(int(ray_off_oracle[-1]), np.int64)
    for r in range(B):
        p = int(ray_off_oracle[r])
        for s in range(3):
            n = int(seg_n[r, s])
            if n:
                idx[p:p + n] = int(seg_off[r, s]) + np.arange(n)
                p += n
    return idx


def gpu_sample(ctx, case, sp, cap=None):
    """snk_sample_segments of the case's pixels with sampler sp; host copies of every output."""
    import ctypes
    import torch
    from paper_2507_01631_b300 import snk
    w = case.w
    B = len(case.pix)
    nseg = 1 + (w.nx == 2) + (w.ny == 2)
    if cap is None:
        cap = B * max(nseg * w.K_max, w.K_ray) + 512
    f32, i32, u8 = torch.float32, torch.int32, torch.uint8
    g = {k: torch.zeros(n, dtype=t, device="cuda") for k, n, t in
         [("ray_od", 6 * B, f32), ("ray_ok", B, u8), ("seg_slot", 3 * B, u8), ("seg_t", 6 * B, f32),
          ("seg_n", 3 * B, i32), ("seg_off", 3 * B, i32), ("smp_t", cap, f32), ("smp_dt", cap, f32),
          ("smp_xyz", 3 * cap, f32), ("state", snk.STATE_WORDS, i32)]}
    pix = torch.from_numpy(np.ascontiguousarray(case.pix.view(np.int32))).cuda()
    ctx.call("snk_sample_segments", ctypes.byref(snk.window_struct(w.window())), snk.ptr(pix), B, ctypes.byref(sp),
             *[snk.ptr(g[k]) for k in ("ray_od", "ray_ok", "seg_slot", "seg_t", "seg_n", "seg_off", "smp_t",
                                       "smp_dt", "smp_xyz")], cap, snk.ptr(g["state"]), None)
    torch.cuda.synchronize()
    h = {k: v.cpu().numpy() for k, v in g.items()}
    h["n_samples"] = int(h["state"][3:4].view(np.uint32)[0])
    return h


# ---- ReLU decisions that binary32 may take either way (mixed path) ----------------
AMBIGUOUS = 1e-6  # |z| / sum|w x| below which a ReLU decision may go either way in binary32


def mask_flip_deltas(case, ref, wc):
    """Changes of the flat FP64 gradient caused by flipping one ambiguous ReLU
    decision (a hidden pre-activation within binary32 rounding of zero).  The
    forward does not move (the unit's activation is ~0 either way); only that
    sample's backward through the unit does, so each flip is one sample's
    contribution recomputed with the other mask, and flips in different samples
    add up."""
    from oracle import hashgrid, mlp, viewdir
    cfg = case.cfg
    smp = ref.smp
    tiles, cols = OS.unflatten(cfg, wc)
    lay = cfg.grid()
    deltas = []
    for k in range(cfg.n_slots):
        idx = np.flatnonzero(smp.slot == k)
        if idx.size == 0:
            continue
        col = (cols[0] if cfg.shared_colour else cols[k]) if cfg.colour else None
        feat = hashgrid.encode(smp.xyz[idx], tiles[k][0], lay)
        sh = viewdir.sh16(ref.extra["d"][smp.ray[idx]].astype(np.float64)) if (cfg.view_dirs and col is not None) else None
        _, _, acts = mlp.forward(feat, tiles[k][1], col, sh)
        layers = [("geo_pre", 0, acts["x0"], tiles[k][1][0]), ("geo_pre", 1, np.maximum(acts["geo_pre"][0], 0), tiles[k][1][1])]
        if col is not None:
            layers += [("col_pre", 0, acts.get("col_in", acts["g"]), col[0]),
                       ("col_pre", 1, np.maximum(acts["col_pre"][0], 0), col[1])]
        for key, li, h, Wm in layers:
            z = acts[key][li]
            ratio = np.abs(z) / (np.abs(h) @ np.abs(Wm).T + 1e-300)
            for s, j in zip(*np.nonzero(ratio < AMBIGUOUS)):
                one = {kk: ([a[s:s + 1].copy() for a in v] if isinstance(v, list) else
                            (v[s:s + 1].copy() if isinstance(v, np.ndarray) else v)) for kk, v in acts.items()}
                flip = {kk: ([a.copy() for a in v] if isinstance(v, list) else
                             (v.copy() if isinstance(v, np.ndarray) else v)) for kk, v in one.items()}
                flip[key][li][0, j] = -flip[key][li][0, j] if flip[key][li][0, j] != 0 else -1e-30
                ds, dr = ref.dsigma[idx[s]:idx[s] + 1], ref.drgb[idx[s]:idx[s] + 1]
                g0 = mlp.backward(ds, dr, tiles[k][1], col, one)
                g1 = mlp.backward(ds, dr, tiles[k][1], col, flip)
                d = np.zeros(cfg.n_params())
                dt, dc = OS.unflatten(cfg, d)
                for q in range(3):
                    dt[k][1][q] += g1[0][q] - g0[0][q]
                    if col is not None:
                        (dc[0] if cfg.shared_colour else dc[k])[q] += g1[1][q] - g0[1][q]
                dt[k][0][...] += hashgrid.encode_backward(smp.xyz[idx[s]:idx[s] + 1], g1[2] - g0[2], lay)
                deltas.append(d)
    return deltas


MAX_FLIPS = 8  # accepted flips per step: a binary32 decision flips only within ~1e-7 of zero
FLIP_FLOOR = GRAD_REL_MIXED / 100  # flips smaller than this (relative to |m|) cannot matter at the tolerance


def flip_groups(cfg):
    """The index ranges the gradient tolerance is applied to: each optimiser's table and MLP part."""
    out = []
    for a, b, mlp_a in OS.group_ranges(cfg):
        if mlp_a > a:
            out.append((a, mlp_a))
        out.append((mlp_a, b))
    return out


def explain_with_flips(got, want, deltas, groups):
    """Greedily add the flip deltas that bring `want` closer to `got`.  Returns the
    adjusted reference and the sizes of the accepted deltas, each relative to |want| in the
    group (flip_groups) where the delta weighs most.  Deltas below FLIP_FLOOR there are left
    out: even a hundred of them could not move a group's norm-wise error across the 5e-3
    tolerance, and whether one brings `want` closer is noise.  The reference may move only by
    exact oracle flips of decisions that are ambiguous in binary32, and by at most MAX_FLIPS of
    them (asserted by the caller)."""
    want = want.copy()
    norms = [max(np.linalg.norm(want[a:b]), 1e-300) for a, b in groups]
    accepted = []
    for d in deltas:
        size = max(float(np.linalg.norm(d[a:b]) / n) for (a, b), n in zip(groups, norms))
        if size < FLIP_FLOOR:
            continue
        if np.linalg.norm(got - (want + d)) < np.linalg.norm(got - want):
            want = want + d
            accepted.append(size)
    return want, accepted
