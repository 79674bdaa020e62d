"""Ray/box clipping, 2x2-window acceptance and the segmented sampler (oracle).
Test infrastructure only.

Paper basis:
* Sec. 4.2 - tiles form a square grid in (East, North); all tiles share
  z_min / z_max; samples are mapped to [0, 1]^3 of their tile.
* Sec. 4.4 - a ray crosses at most 3 tiles; rays are accepted only if every
  tile they cross is loaded (in the window), others are rejected.
* Sec. 4.5 - per tile the ray gets its own near/far pair (N_i, F_i) so that
  segment ends fall exactly on tile faces; each segment is sampled
  separately; the face point belongs to both neighbouring segments.

Readings where the paper is silent:
* acceptance = the ray's intersection with the scene box is non-empty and
  contained in its intersection with the window box;
* segments split the scene-box interval at the interior planes of the window;
  zero-length pieces are dropped; a segment's tile is the tile holding its
  midpoint (ties go to the lower tile index);
* samples per segment K = clamp(rint(K_ray * len_seg / len_ray), K_min, K_max)
  (round half to even);
* stratified bins: K equal bins of width w = len/K; sample k at
  t0 + (k + u_k) w with u_k uniform (0.5 when rendering); its delta is w
  (bin convention of Nerfstudio, on which the paper builds, Sec. 4.6).
  With this convention the deltas of a ray add up to its box-intersection
  length and the face point gets no double weight.

Two variants for comparisons (sampler modes):
* UNIFORM, the NeRF-XL distribution the paper contrasts with its own (Sec.
  4.5): K_ray bins over the whole scene interval [t_in, t_out], sample j at
  t_in + (j + u_j) w; each sample belongs to the tile holding its point (a
  point on an interior plane goes to the lower tile) and the samples of a tile
  form its segment; delta = w.
* POINTS, point samples (the setting of the paper's remark that the face
  point, sampled as F_1 and again as N_2, has its N_2 density ignored): K
  points per segment at t0 + k (t1 - t0) / (K - 1), the last exactly at t1,
  with delta_i = t_i - t_{i-1} along the ray (0 for the ray's first point).

Every float that decides something discrete (the slab parameters, the
segment bounds, K, sample positions and local coordinates) is *defined* as
the binary32 operation sequence written below (each numpy float32 op rounds
once, no fused multiply-add).
"""

SEGMENTS, UNIFORM, POINTS = 0, 1, 2
from dataclasses import dataclass
import numpy as np

from . import philox

F32 = np.float32


@dataclass
class WindowF32:
    """Binary32 constants of a window, derived from the FP64 window description
    by correctly rounded conversion (the library does the same)."""
    nx: int
    ny: int
    win_hi: np.ndarray        # (3,) float32: nx*Wt, ny*Ht, Z
    scene_lo: np.ndarray      # (3,) float32, window-local
    scene_hi: np.ndarray
    split: np.ndarray         # (2,) float32: Wt, Ht  (interior planes)
    tile_size: np.ndarray     # (3,) float32
    inv_size: np.ndarray      # (3,) float32: 1/Wt, 1/Ht, 1/Z rounded from FP64
    slot: tuple


def window_f32(win):
    o = np.asarray(win.origin, np.float64)
    ts = np.asarray(win.tile_size, np.float64)
    win_hi = np.array([win.nx * ts[0], win.ny * ts[1], ts[2]], np.float64).astype(F32)
    s_lo = (np.asarray(win.scene_lo, np.float64) - o).astype(F32)
    s_hi = (np.asarray(win.scene_hi, np.float64) - o).astype(F32)
    return WindowF32(win.nx, win.ny, win_hi, s_lo, s_hi, ts[:2].astype(F32), ts.astype(F32),
                     (1.0 / ts).astype(F32), tuple(win.slot))


def slab(o, d, lo, hi):
    """Slab-method clip of rays (o, d) (float32 (n, 3)) to the box [lo, hi].
    Returns float32 (t_in, t_out) and the binary32 reciprocals inv (n, 3).
    Per axis: inv = 1/d; t1 = (lo - o) * inv; t2 = (hi - o) * inv; near/far =
    min/max.  An axis with d == 0 gives (-inf, +inf) if lo <= o <= hi and
    (+inf, -inf) otherwise.  t_in = max(0, near_x, near_y, near_z),
    t_out = min(far_x, far_y, far_z); the ray hits iff t_in < t_out."""
    n = o.shape[0]
    tn = np.zeros((n, 3), F32)
    tf = np.zeros((n, 3), F32)
    inv = np.zeros((n, 3), F32)
    for a in range(3):
        da = d[:, a]
        zero = da == 0
        with np.errstate(divide="ignore", invalid="ignore"):
            ia = np.where(zero, F32(np.inf), F32(1.0) / np.where(zero, F32(1.0), da)).astype(F32)
        inv[:, a] = ia
        with np.errstate(invalid="ignore"):
            t1 = ((F32(lo[a]) - o[:, a]).astype(F32) * ia).astype(F32)
            t2 = ((F32(hi[a]) - o[:, a]).astype(F32) * ia).astype(F32)
        near = np.minimum(t1, t2)
        far = np.maximum(t1, t2)
        inside = (o[:, a] >= F32(lo[a])) & (o[:, a] <= F32(hi[a]))
        near = np.where(zero, np.where(inside, F32(-np.inf), F32(np.inf)), near)
        far = np.where(zero, np.where(inside, F32(np.inf), F32(-np.inf)), far)
        tn[:, a] = near
        tf[:, a] = far
    t_in = np.maximum(np.maximum(np.maximum(F32(0.0), tn[:, 0]), tn[:, 1]), tn[:, 2]).astype(F32)
    t_out = np.minimum(np.minimum(tf[:, 0], tf[:, 1]), tf[:, 2]).astype(F32)
    return t_in, t_out, inv


@dataclass
class Segments:
    ray_ok: np.ndarray      # (B,) uint8
    t_in: np.ndarray        # (B,) float32 scene-box entry (0 if rejected)
    t_out: np.ndarray       # (B,) float32
    n_seg: np.ndarray       # (B,) int
    slot: np.ndarray        # (B, 3) int (255 if unused)
    t0: np.ndarray          # (B, 3) float32
    t1: np.ndarray          # (B, 3) float32
    K: np.ndarray           # (B, 3) int samples per segment (0 if unused)
    ray_off: np.ndarray     # (B+1,) int64 CSR of samples per ray


def accepted(o, d, wf):
    """Sec. 4.4 acceptance of every ray: its scene-box interval is non-empty and lies
    inside the window box.  Returns (ok, ts_in, ts_out, inv)."""
    zero3 = np.zeros(3, F32)
    ts_in, ts_out, inv = slab(o, d, wf.scene_lo, wf.scene_hi)
    tw_in, tw_out, _ = slab(o, d, zero3, wf.win_hi)
    hit = ts_in < ts_out
    return hit & (tw_in <= ts_in) & (ts_out <= tw_out), ts_in, ts_out, inv


def segments(o, d, wf, K_ray, K_min, K_max):
    """Acceptance test and segment split for every ray; see module docstring."""
    B = o.shape[0]
    ok, ts_in, ts_out, inv = accepted(o, d, wf)

    n_seg = np.zeros(B, np.int64)
    slot = np.full((B, 3), 255, np.int64)
    t0 = np.zeros((B, 3), F32)
    t1 = np.zeros((B, 3), F32)
    K = np.zeros((B, 3), np.int64)
    for i in range(B):
        if not ok[i]:
            continue
        a, b = ts_in[i], ts_out[i]
        cuts = []
        for axis, nsplit in ((0, wf.nx), (1, wf.ny)):
            if nsplit == 2 and d[i, axis] != 0:
                tp = F32(F32(wf.split[axis] - o[i, axis]) * inv[i, axis])
                if a < tp < b:
                    cuts.append(tp)
        bounds = [a] + sorted(cuts) + [b]
        len_ray = F32(b - a)
        s = 0
        for j in range(len(bounds) - 1):
            lo_t, hi_t = bounds[j], bounds[j + 1]
            if not (hi_t - lo_t > 0):
                continue
            mid = F32(lo_t + F32(F32(hi_t - lo_t) * F32(0.5)))
            ix = 1 if (wf.nx == 2 and F32(o[i, 0] + F32(mid * d[i, 0])) > wf.split[0]) else 0
            iy = 1 if (wf.ny == 2 and F32(o[i, 1] + F32(mid * d[i, 1])) > wf.split[1]) else 0
            len_seg = F32(hi_t - lo_t)
            q = F32(len_seg / len_ray)
            kf = F32(F32(K_ray) * q)
            k = int(np.rint(kf))
            k = min(max(k, K_min), K_max)
            slot[i, s] = wf.slot[iy * wf.nx + ix]
            t0[i, s] = lo_t
            t1[i, s] = hi_t
            K[i, s] = k
            s += 1
        n_seg[i] = s
    per_ray = K.sum(axis=1)
    ray_off = np.zeros(B + 1, np.int64)
    ray_off[1:] = np.cumsum(per_ray)
    return Segments(ok.astype(np.uint8), np.where(ok, ts_in, F32(0)), np.where(ok, ts_out, F32(0)),
                    n_seg, slot, t0, t1, K, ray_off)


def _uniform_t(a, w, seed, iteration, rid, j, render):
    """t of sample j of a ray in the NeRF-XL distribution (binary32)."""
    j = np.asarray(j)
    u = np.full(j.shape, F32(0.5), F32) if render else philox.jitter(seed, iteration, rid, j).astype(F32)
    return (a + ((j.astype(F32) + u).astype(F32) * w).astype(F32)).astype(F32)


def segments_uniform(o, d, wf, K_ray, seed, iteration, render=False, ray_ids=None):
    """NeRF-XL distribution: the segments are the runs of same-tile samples (see
    module docstring); each segment's (t0, t1) is the ray's (t_in, t_out)."""
    B = o.shape[0]
    ok, ts_in, ts_out, inv = accepted(o, d, wf)
    n_seg = np.zeros(B, np.int64)
    slot = np.full((B, 3), 255, np.int64)
    t0 = np.zeros((B, 3), F32)
    t1 = np.zeros((B, 3), F32)
    K = np.zeros((B, 3), np.int64)
    for i in range(B):
        if not ok[i]:
            continue
        a, b = ts_in[i], ts_out[i]
        w = F32(F32(b - a) / F32(K_ray))
        rid = i if ray_ids is None else int(ray_ids[i])
        t = _uniform_t(a, w, seed, iteration, rid, np.arange(K_ray), render)
        ix = (wf.nx == 2) & ((o[i, 0] + (t * d[i, 0]).astype(F32)).astype(F32) > wf.split[0])
        iy = (wf.ny == 2) & ((o[i, 1] + (t * d[i, 1]).astype(F32)).astype(F32) > wf.split[1])
        tile = iy.astype(np.int64) * wf.nx + ix.astype(np.int64)
        s = -1
        for j in range(K_ray):
            if j == 0 or tile[j] != tile[j - 1]:
                s += 1
                slot[i, s] = wf.slot[tile[j]]
                t0[i, s], t1[i, s] = a, b
            K[i, s] += 1
        n_seg[i] = s + 1
    ray_off = np.zeros(B + 1, np.int64)
    ray_off[1:] = np.cumsum(K.sum(axis=1))
    return Segments(ok.astype(np.uint8), np.where(ok, ts_in, F32(0)), np.where(ok, ts_out, F32(0)),
                    n_seg, slot, t0, t1, K, ray_off)


@dataclass
class Samples:
    ray: np.ndarray     # (S,) int64 ray index of each sample
    slot: np.ndarray    # (S,) int64 parameter slot
    t: np.ndarray       # (S,) float32
    dt: np.ndarray      # (S,) float32
    xyz: np.ndarray     # (S, 3) float32 tile-local coordinates in [0, 1]


def stratified(o, d, seg, wf, seed, iteration, render=False, ray_ids=None, mode=SEGMENTS):
    """Sample positions of every segment (see module docstring).  `ray_ids`
    gives each ray's index in its batch (the jitter counter); default 0..B-1.
    Sample k of a segment [t0, t1] with K bins of width w = (t1 - t0) / K sits
    at t = t0 + (k + u) * w, u = jitter of its index along the ray (0.5 when
    rendering); world point p = o + t d; tile-local l = clamp((p - tile_lo) *
    inv_size, 0, 1)."""
    rays_l, slot_l, t_l, dt_l, xyz_l = [], [], [], [], []
    B = o.shape[0]
    for i in range(B):
        j0 = 0
        t_last = None
        for s in range(seg.n_seg[i]):
            k_n = int(seg.K[i, s])
            a, b = seg.t0[i, s], seg.t1[i, s]
            k = np.arange(k_n)
            rid = i if ray_ids is None else int(ray_ids[i])
            if mode == UNIFORM:
                w = F32(F32(b - a) / F32(sum(int(x) for x in seg.K[i])))
                t = _uniform_t(a, w, seed, iteration, rid, j0 + k, render)
                dt = np.full(k_n, w, F32)
            elif mode == POINTS:
                w = F32(F32(b - a) / F32(k_n - 1))
                t = (a + (k.astype(F32) * w).astype(F32)).astype(F32)
                t[-1] = b
                prev = np.concatenate([[t[0] if t_last is None else t_last], t[:-1]]).astype(F32)
                dt = (t - prev).astype(F32)
                t_last = b
            else:
                w = F32(F32(b - a) / F32(k_n))
                if render:
                    u = np.full(k_n, F32(0.5), F32)
                else:
                    u = philox.jitter(seed, iteration, rid, j0 + k).astype(F32)
                t = (a + ((k.astype(F32) + u).astype(F32) * w).astype(F32)).astype(F32)
                dt = np.full(k_n, w, F32)
            sl = int(seg.slot[i, s])
            tile = wf.slot.index(sl)
            ix, iy = tile % wf.nx, tile // wf.nx
            # tile lower corner in window-local binary32: (ix * Wt, iy * Ht, 0), ix, iy in {0, 1}
            lo = np.array([F32(ix) * wf.split[0] if ix else F32(0), F32(iy) * wf.split[1] if iy else F32(0),
                           F32(0)], F32)
            p = (o[i][None, :] + (t[:, None] * d[i][None, :]).astype(F32)).astype(F32)
            loc = ((p - lo[None, :]).astype(F32) * wf.inv_size[None, :]).astype(F32)
            loc = np.minimum(np.maximum(loc, F32(0)), F32(1))
            rays_l.append(np.full(k_n, i))
            slot_l.append(np.full(k_n, sl))
            t_l.append(t)
            dt_l.append(dt)
            xyz_l.append(loc)
            j0 += k_n
    if not rays_l:
        e = np.zeros(0)
        return Samples(e.astype(np.int64), e.astype(np.int64), e.astype(F32), e.astype(F32), np.zeros((0, 3), F32))
    return Samples(np.concatenate(rays_l), np.concatenate(slot_l), np.concatenate(t_l),
                   np.concatenate(dt_l), np.concatenate(xyz_l))
