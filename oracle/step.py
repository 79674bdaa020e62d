"""One training step and one render call of the per-tile / 2x2-window NeRF
(oracle, FP64).  Test infrastructure only.

The step follows the paper's procedure for a batch of rays (Sec. 4.4, last
paragraph; Sec. 4.5): rays from the cameras (camera.py), acceptance and
segmented sampling (sampler.py), per-sample NGP encoding with the sample's
tile table (hashgrid.py), the tile's density MLP and the colour MLP (mlp.py),
volume rendering and the colour loss (render.py), the backward pass, and an
Adam update per optimiser (adam.py): one per tile (its table and density
MLP) and one for the colour MLP (shared) or one per tile colour MLP.

Flat parameter layout (also the library's):
    [slot 0 | slot 1 | ... | slot n-1 | colour 0 (| colour 1 ...)]
    slot block   = table (n_entries x F, entry-major) | W1 | W2 | W3
    colour block = V1 | V2 | V3        (each matrix row-major [out][in])
"""
from dataclasses import dataclass, field
import numpy as np

from . import adam, camera, hashgrid, mlp, occupancy, quant, render, sampler, viewdir


@dataclass
class ModelConfig:
    L: int = 8
    F: int = 2
    log2_T: int = 14
    n_min: int = 16
    n_max: int = 256
    hidden: int = 64
    geo_out: int = 4            # 4: no colour net; 16: with colour net
    colour: bool = False
    shared_colour: bool = True
    n_slots: int = 1
    K_ray: int = 64
    K_min: int = 64
    K_max: int = 64
    first_layer: str = "f16"    # "e4m3": the density MLP's input is quantised (quant.py)
    view_dirs: bool = False     # colour input [g | SH_16(ray direction)] (viewdir.py)

    def grid(self):
        return hashgrid.layout(self.L, self.F, self.log2_T, self.n_min, self.n_max)

    def geo_shapes(self):
        return [(self.hidden, self.L * self.F), (self.hidden, self.hidden), (self.geo_out, self.hidden)]

    def col_shapes(self):
        cin = self.geo_out + (16 if self.view_dirs else 0)
        return [(self.hidden, cin), (self.hidden, self.hidden), (3, self.hidden)] if self.colour else []

    def tile_params(self):
        return self.grid().n_params + sum(a * b for a, b in self.geo_shapes())

    def col_params(self):
        return sum(a * b for a, b in self.col_shapes())

    def n_colour_blocks(self):
        if not self.colour:
            return 0
        return 1 if self.shared_colour else self.n_slots

    def n_params(self):
        return self.n_slots * self.tile_params() + self.n_colour_blocks() * self.col_params()

    def n_optimisers(self):
        return self.n_slots + self.n_colour_blocks()


def _mats(flat, start, shapes):
    out = []
    p = start
    for a, b in shapes:
        out.append(flat[p:p + a * b].reshape(a, b))
        p += a * b
    return out, p


def unflatten(cfg, flat):
    """Views into flat: list over slots of (table, [W1, W2, W3]) and the list of
    colour blocks [V1, V2, V3]."""
    lay = cfg.grid()
    tiles = []
    p = 0
    for _ in range(cfg.n_slots):
        table = flat[p:p + lay.n_params].reshape(lay.n_entries, cfg.F)
        p += lay.n_params
        geo, p = _mats(flat, p, cfg.geo_shapes())
        tiles.append((table, geo))
    cols = []
    for _ in range(cfg.n_colour_blocks()):
        c, p = _mats(flat, p, cfg.col_shapes())
        cols.append(c)
    return tiles, cols


def group_ranges(cfg):
    """(start, end, mlp_start) of every optimiser's parameters in the flat
    vector; entries from mlp_start on get the L2 weight decay."""
    lay = cfg.grid()
    out = []
    for s in range(cfg.n_slots):
        a = s * cfg.tile_params()
        out.append((a, a + cfg.tile_params(), a + lay.n_params))
    base = cfg.n_slots * cfg.tile_params()
    for c in range(cfg.n_colour_blocks()):
        a = base + c * cfg.col_params()
        out.append((a, a + cfg.col_params(), a))
    return out


@dataclass
class StepResult:
    seg: sampler.Segments
    smp: sampler.Samples
    sigma: np.ndarray
    rgb_s: np.ndarray
    rgb: np.ndarray
    depth: np.ndarray
    opacity: np.ndarray
    t_final: np.ndarray
    loss: float = 0.0
    grad: np.ndarray = None
    dsigma: np.ndarray = None
    drgb: np.ndarray = None
    params: np.ndarray = None
    m: np.ndarray = None
    v: np.ndarray = None
    extra: dict = field(default_factory=dict)


def sample_rays(cfg, cameras, win, pix, seed, iteration, render_mode, ray_ids=None, occ=None, mode=0):
    """occ: (occupied flags (n_slots, R^3), R) to cull samples in empty cells, or None;
    mode: sampler.SEGMENTS (the paper's), UNIFORM (NeRF-XL) or POINTS."""
    o, d = camera.rays(cameras, pix, win.origin, win.origin[2], win.origin[2] + win.tile_size[2])
    wf = sampler.window_f32(win)
    if mode == sampler.UNIFORM:
        seg = sampler.segments_uniform(o, d, wf, cfg.K_ray, seed, iteration, render=render_mode, ray_ids=ray_ids)
    else:
        seg = sampler.segments(o, d, wf, cfg.K_ray, cfg.K_min, cfg.K_max)
    smp = sampler.stratified(o, d, seg, wf, seed, iteration, render=render_mode, ray_ids=ray_ids, mode=mode)
    if occ is not None:
        seg, smp = occupancy.cull(seg, smp, occ[0], occ[1])
    return o, d, seg, smp


def field_forward(cfg, flat, smp, dirs=None):
    """sigma (S,), rgb (S, 3) and per-slot activations.  dirs (B, 3): the rays'
    unit directions (binary32), needed by the view-direction colour input."""
    lay = cfg.grid()
    tiles, cols = unflatten(cfg, flat)
    S = len(smp.t)
    sigma = np.zeros(S)
    rgb = np.zeros((S, 3))
    saved = {}
    for s in range(cfg.n_slots):
        m = smp.slot == s
        if not m.any():
            continue
        table, geo = tiles[s]
        feat = hashgrid.encode(smp.xyz[m], table, lay)
        scale = None
        if cfg.first_layer == "e4m3":
            # per-tensor scale of this slot's first-layer input from the current batch; the codes
            # are decided in binary32 (the kernel's precision), the MLP sees scale x value(code)
            # and its backward passes dfeat straight through the quantiser
            f32 = quant.encode_binary32(smp.xyz[m], table, lay)
            scale = quant.slot_scale_binary32(f32)
            feat = quant.quantise_binary32(f32, scale)
        col = None
        if cfg.colour:
            col = cols[0] if cfg.shared_colour else cols[s]
        sh = viewdir.sh16(dirs[smp.ray[m]].astype(np.float64)) if (cfg.view_dirs and col is not None) else None
        sg, rg, acts = mlp.forward(feat, geo, col, sh)
        sigma[m] = sg
        rgb[m] = rg
        acts["scale"] = scale
        saved[s] = (m, feat, acts, col)
    return sigma, rgb, saved


def train_step(cfg, flat, m_state, v_state, steps, cameras, win, pix, targets, seed, iteration, lr=None, occ=None,
               mode=0):
    """One training step.  targets: list of per-view crop images (h, w, 3).
    steps: per-optimiser Adam step counts before this step (updated copy is
    returned in extra["steps"]).  lr: Adam learning rate (I-NGP's 1e-2 unless given).
    occ: (occupied flags, R) of the slots' occupancy grids to cull samples, or None."""
    o, d, seg, smp = sample_rays(cfg, cameras, win, pix, seed, iteration, False, occ=occ, mode=mode)
    sigma, rgb_s, saved = field_forward(cfg, flat, smp, dirs=d)
    rgb, depth, opac, tfin, _ = render.composite(sigma, rgb_s, smp.t.astype(np.float64),
                                                 smp.dt.astype(np.float64), seg.ray_off)
    gt = gather_targets(cameras, pix, targets)
    loss, g_rgb = render.mse_loss(rgb, gt, seg.ray_ok)
    dsigma, drgb = render.composite_backward(g_rgb, sigma, rgb_s, smp.t.astype(np.float64),
                                             smp.dt.astype(np.float64), seg.ray_off)
    grad = np.zeros_like(flat)
    gtiles, gcols = unflatten(cfg, grad)
    lay = cfg.grid()
    tiles, cols = unflatten(cfg, flat)
    for s, (m, feat, acts, col) in saved.items():
        dgeo, dcol, dfeat = mlp.backward(dsigma[m], drgb[m], tiles[s][1], col, acts)
        for k in range(3):
            gtiles[s][1][k] += dgeo[k]
        if cfg.colour:
            tgt = gcols[0] if cfg.shared_colour else gcols[s]
            for k in range(3):
                tgt[k] += dcol[k]
        gtiles[s][0][...] += hashgrid.encode_backward(smp.xyz[m], dfeat, lay)
    new = flat.copy()
    m_new = m_state.copy()
    v_new = v_state.copy()
    steps = list(steps)
    for gi, (a, b, mlp_a) in enumerate(group_ranges(cfg)):
        steps[gi] += 1
        l2 = np.zeros(b - a)
        l2[mlp_a - a:] = adam.L2_MLP
        w, mm, vv = adam.step(flat[a:b], grad[a:b], m_state[a:b], v_state[a:b], steps[gi],
                              lr=adam.LR if lr is None else lr, l2=l2)
        new[a:b], m_new[a:b], v_new[a:b] = w, mm, vv
    res = StepResult(seg, smp, sigma, rgb_s, rgb, depth, opac, tfin, loss, grad, dsigma, drgb, new, m_new, v_new)
    res.extra["steps"] = steps
    res.extra["o"], res.extra["d"] = o, d
    res.extra["gt"] = gt
    return res


def render_rays(cfg, flat, cameras, win, pix, seed=0, iteration=0, render_mode=True, ray_ids=None, occ=None,
                mode=0):
    """Forward only: per-ray rgb, depth, opacity (bin-centre samples unless
    render_mode is False, then the training jitter of the given ray ids)."""
    o, d, seg, smp = sample_rays(cfg, cameras, win, pix, seed, iteration, render_mode, ray_ids, occ=occ, mode=mode)
    sigma, rgb_s, _ = field_forward(cfg, flat, smp, dirs=d)
    rgb, depth, opac, tfin, _ = render.composite(sigma, rgb_s, smp.t.astype(np.float64),
                                                 smp.dt.astype(np.float64), seg.ray_off)
    res = StepResult(seg, smp, sigma, rgb_s, rgb, depth, opac, tfin)
    res.extra["o"], res.extra["d"] = o, d
    return res


def gather_targets(cameras, pix, targets):
    """Target colour of each packed pixel from its view's resident crop."""
    from synth import unpack_pixel
    v, r, c = unpack_pixel(pix)
    out = np.zeros((len(v), 3))
    for i in range(len(v)):
        r0, c0, h, w = cameras[v[i]].crop
        out[i] = targets[v[i]][r[i] - r0, c[i] - c0]
    return out
