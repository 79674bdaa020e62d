"""Snake sweep of a tile grid on one GPU (Sec. 4.4): a 2 x 2 window slides
over the grid in snake order; only the window's four tiles are resident in
the model's four parameter slots, every other tile's trainable state
(parameters, FP16 working copy, Adam moments and step count) is parked in
pinned host memory, and the colour network stays resident.

A move keeps two tiles in their slots and exchanges the other two.  The
exchange overlaps training: while the window trains at one position, a copy
stream brings the next position's two entering tiles from host memory into
device staging blocks; at the move the leaving tiles are parked into two
other staging blocks and the entering ones unparked into the freed slots
(device-to-device copies through snk_tile_park / snk_tile_unpark), and the
copy stream then writes the leaving tiles back to host memory during the
next position's training.  Only the two device-to-device exchanges are on
the training stream.

Host logic only: every step runs through snk_train_step, every tile copy
through the library or a stream copy.
"""
import argparse
import ctypes
import json
import os
import sys
import time

import numpy as np
import torch

from . import snk
from .trainer import Trainer, model_from_workload


def snake_order(gx, gy):
    """Window positions (lower-left tile) over a gx x gy tile grid: along the
    first row of positions, then each next row in the opposite direction."""
    out = []
    for row in range(gy - 1):
        cols = list(range(gx - 1))
        out += [(c, row) for c in (cols if row % 2 == 0 else cols[::-1])]
    return out


def window_members(pos):
    """The grid tiles of the window at pos, in window order (ix + 2 iy)."""
    x, y = pos
    return [(x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1)]


def exchanges(order):
    """For every move: (leaving tiles, entering tiles), two each."""
    out = []
    for a, b in zip(order[:-1], order[1:]):
        ta, tb = window_members(a), window_members(b)
        out.append(([t for t in ta if t not in tb], [t for t in tb if t not in ta]))
    return out


class SnakeSweep:
    """The tile states of a grid and the resident window of one model."""

    def __init__(self, ctx, workload, tile_init, colour_init, precision=None, sampler=None, adam=None,
                 loss_scale=None, device="cuda"):
        self.ctx = ctx
        self.w = workload
        self.grid = workload.grid_tiles()
        self.model = model_from_workload(workload, precision)
        self.lay = snk.layout(self.model)
        w = workload
        self.sampler = sampler or snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 1, 0)
        nt = self.lay.tile_params
        init = np.concatenate([np.asarray(tile_init((0, 0)), np.float32)] * 4 + [np.asarray(colour_init, np.float32)])
        self.tr = Trainer(ctx, self.model, snk.window_struct(w.window()), self.sampler, init, adam=adam,
                          loss_scale=loss_scale, device=device)
        nb = ctypes.c_int64()
        snk.check(snk.load().snk_tile_bytes(ctypes.byref(self.model), ctypes.byref(nb)))
        self.tile_bytes = nb.value
        self.host = {}
        self.staging_in = [torch.empty(self.tile_bytes, dtype=torch.uint8, device=device) for _ in range(2)]
        self.staging_out = [torch.empty(self.tile_bytes, dtype=torch.uint8, device=device) for _ in range(2)]
        # every tile's initial state, laid out by the library: write it into slot 0, park it
        tr = self.tr
        for iy in range(self.grid[1]):
            for ix in range(self.grid[0]):
                t = (ix, iy)
                tr.params[:nt] = torch.as_tensor(np.asarray(tile_init(t), np.float32), device=device)
                if tr.params_lp is not None:
                    tr.params_lp[:nt] = tr.params[:nt].to(torch.float16).view(torch.int16)
                tr.m[:nt] = 0
                tr.v[:nt] = 0
                tr.steps[0] = 0
                self.host[t] = torch.empty(self.tile_bytes, dtype=torch.uint8, pin_memory=True)
                self._park(0, self.host[t], None)
        torch.cuda.synchronize()
        self.slot_of = {}

    def _park(self, slot, dst, stream):
        self.ctx.call("snk_tile_park", ctypes.byref(self.model), ctypes.byref(self.tr.p_struct), slot, snk.ptr(dst),
                      snk.stream_handle(stream))

    def _unpark(self, slot, src, stream):
        self.ctx.call("snk_tile_unpark", ctypes.byref(self.model), ctypes.byref(self.tr.p_struct), slot, snk.ptr(src),
                      snk.stream_handle(stream))

    def window_at(self, pos):
        slots = [self.slot_of[t] for t in window_members(pos)]
        return snk.window_struct(self.w.window(pos, slot=slots))


    def run(self, iters, batch_at, views_at=None, on_step=None):
        """Train `iters` steps at every position of the snake order.
        batch_at(pos, i) -> int32 device pixels; views_at(pos) (optional) sets the
        context's views for the position; on_step(pos, i, out) sees the rendered
        [B][5] output of every step.  Returns per-position timings (ms)."""
        main = torch.cuda.current_stream()
        copy = torch.cuda.Stream()
        order = snake_order(*self.grid)
        moves = exchanges(order)
        ev_moved = torch.cuda.Event()
        ev_ready = torch.cuda.Event()
        stats = []
        # the first window: its four tiles into slots 0..3
        self.slot_of = {}
        for k, t in enumerate(window_members(order[0])):
            self._unpark(k, self.host[t], main)
            self.slot_of[t] = k
        for k, pos in enumerate(order):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(main)
            if k > 0:
                leaving, entering = moves[k - 1]
                main.wait_event(ev_ready)  # entering tiles staged, previous write-back done
                for j, (tl, te) in enumerate(zip(leaving, entering)):
                    s = self.slot_of.pop(tl)
                    self._park(s, self.staging_out[j], main)
                    self._unpark(s, self.staging_in[j], main)
                    self.slot_of[te] = s
                ev_moved.record(main)
                copy.wait_event(ev_moved)
                with torch.cuda.stream(copy):
                    for j, tl in enumerate(leaving):
                        self.host[tl].copy_(self.staging_out[j], non_blocking=True)
            e1.record(main)
            if k + 1 < len(order):
                if k == 0:
                    copy.wait_stream(main)
                with torch.cuda.stream(copy):
                    for j, te in enumerate(moves[k][1]):
                        self.staging_in[j].copy_(self.host[te], non_blocking=True)
                ev_ready.record(copy)
            if views_at is not None:
                views_at(pos)
            self.tr.window = self.window_at(pos)
            for i in range(iters):
                pix = batch_at(pos, i)
                if on_step is not None:
                    out = torch.zeros(pix.numel() * 5, dtype=torch.float32, device=pix.device)
                    self.tr.train_step(pix, out, stream=main)
                    on_step(pos, i, out)
                else:
                    self.tr.train_step(pix, stream=main)
            e2.record(main)
            stats.append((pos, e0, e1, e2))
        # park the last window back to host memory
        for t, s in self.slot_of.items():
            self._park(s, self.host[t], main)
        torch.cuda.synchronize()
        return [{"pos": list(p), "move_ms": a.elapsed_time(b), "train_ms": b.elapsed_time(c)} for p, a, b, c in stats]

    def tile_state(self, t):
        """(params, m, v, step) of tile t, read back through slot 0 (use after run())."""
        nt = self.lay.tile_params
        self._unpark(0, self.host[t], None)
        torch.cuda.synchronize()
        tr = self.tr
        return (tr.params[:nt].cpu().numpy(), tr.m[:nt].cpu().numpy(), tr.v[:nt].cpu().numpy(),
                int(tr.steps[0].item()))


class DeviceBatches:
    """Ray batches built on the device (Sec. 4.3 crops, Sec. 4.4 acceptance): per
    window position the crops of its tiles in every view (snk_build_crops), the
    accepted pixels of those crops (snk_ray_pool), then one Philox draw per step
    (snk_draw_batch).  The views' resident crops follow the window: set_crops(rects)
    receives the per-view rectangles (host) to load the matching target regions."""

    def __init__(self, ctx, workload, n_views, rays, margin=64, cap=1 << 26, seed=1):
        self.ctx, self.w, self.nv, self.rays, self.margin, self.cap, self.seed = ctx, workload, n_views, rays, margin, cap, seed
        self.tile_rects = torch.zeros(n_views * 16, dtype=torch.int32, device="cuda")
        self.view_rects = torch.zeros(n_views * 4, dtype=torch.int32, device="cuda")
        self.pool = torch.zeros(cap, dtype=torch.int32, device="cuda")
        self.n_pool = torch.zeros(2, dtype=torch.int32, device="cuda")
        self.pix = torch.zeros(rays, dtype=torch.int32, device="cuda")
        self.step = 0

    def position(self, pos, set_crops=None):
        """Crops and pool of the window at pos; returns the view rectangles (host)."""
        ws = snk.window_struct(self.w.window(pos))
        self.ctx.call("snk_build_crops", ctypes.byref(ws), self.margin, snk.ptr(self.tile_rects),
                      snk.ptr(self.view_rects), None)
        rects = self.view_rects.cpu().numpy().reshape(self.nv, 4)
        if set_crops is not None:
            set_crops(rects)
        self.ctx.call("snk_ray_pool", ctypes.byref(ws), snk.ptr(self.view_rects), snk.ptr(self.pool), self.cap,
                      snk.ptr(self.n_pool), None)
        return rects

    def draw(self):
        self.ctx.call("snk_draw_batch", snk.ptr(self.pool), snk.ptr(self.n_pool), self.rays, self.seed, self.step,
                      snk.ptr(self.pix), None)
        self.step += 1
        return self.pix


def _main():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from synth import workloads as W
    import synth
    ap = argparse.ArgumentParser(description="time a snake sweep over a tile grid")
    ap.add_argument("--workload", default="sweep_grid8")
    ap.add_argument("--grid", type=int, nargs="+", default=[3, 4, 5])
    ap.add_argument("--iters", type=int, default=20, help="training steps per window position")
    ap.add_argument("--rays", type=int, default=0)
    ap.add_argument("--device-batches", type=int, default=1,
                    help="1: crops, ray pool and batches built on the device; 0: host-drawn batches")
    args = ap.parse_args()
    from . import build
    build.build()
    ctx = snk.Context(0)
    res = []
    for g in args.grid:
        w = W.get(args.workload, grid=(g, g))
        if args.rays:
            w = W.get(args.workload, grid=(g, g), n_rays=args.rays)
        cams = W.cameras(w)
        model = model_from_workload(w)
        lay = snk.layout(model)
        geo = [(64, w.L * w.F), (64, 64), (w.geo_out, 64)]
        col = [(64, w.geo_out + (16 if w.view_dirs else 0)), (64, 64), (3, 64)]
        p0 = W.init_params(lay.grid_params, geo, col, 1, 1, w.seed)
        tile0, colour0 = p0[:lay.tile_params], p0[lay.tile_params:]
        sw = SnakeSweep(ctx, w, lambda t: tile0, colour0)
        # targets: one device image per view, large enough for any window crop; content does not
        # change the work, so it is a seeded smooth image
        crops_at = {}
        order = snake_order(g, g)
        for pos in order:
            rects = W.tile_crops(w, cams, pos)
            crops_at[pos] = [(min(r[0] for r in rs), min(r[1] for r in rs),
                              max(r[0] + r[2] for r in rs) - min(r[0] for r in rs),
                              max(r[1] + r[3] for r in rs) - min(r[1] for r in rs)) for rs in rects]
        hmax = max(c[2] for cs in crops_at.values() for c in cs)
        wmax = max(c[3] for cs in crops_at.values() for c in cs)
        side = max(hmax, wmax)
        if args.device_batches:  # crops come from the device: an image-sized buffer bounds any of them
            side = max(max(c.height, c.width) for c in cams)
        img = torch.from_numpy(synth.smooth_images(w.seed + 17, 1, side, side)[0]).cuda()
        images = [img for _ in cams]

        def views_at(pos):
            cs = []
            for cam, c in zip(cams, crops_at[pos]):
                cam.crop = c
                cs.append(cam)
            ctx.set_views(cs, images)

        if args.device_batches:
            db = DeviceBatches(ctx, w, len(cams), w.n_rays, margin=w.crop_margin)
            ctx.set_views(cams, images)  # whole-image crops for the first crop build

            def views_at_dev(pos):
                def set_crops(rects):
                    cs = []
                    for cam, r in zip(cams, rects):
                        cam.crop = tuple(int(x) for x in r)
                        cs.append(cam)
                    ctx.set_views(cs, images)
                db.position(pos, set_crops)

            t0 = time.perf_counter()
            stats = sw.run(args.iters, lambda pos, i: db.draw(), views_at=views_at_dev)
        else:
            batches = {pos: [torch.from_numpy(W.batch(w, cams, 50 + i, pos=pos).view(np.int32)).cuda()
                             for i in range(2)] for pos in order}
            t0 = time.perf_counter()
            stats = sw.run(args.iters, lambda pos, i: batches[pos][i % 2], views_at=views_at)
        wall = time.perf_counter() - t0
        st = sw.tr.read_state()
        train = sum(s["train_ms"] for s in stats)
        move = sum(s["move_ms"] for s in stats[1:])
        res.append({"grid": [g, g], "tiles": g * g, "positions": len(order), "iters_per_position": args.iters,
                    "rays_per_iter": w.n_rays, "wall_s": wall, "train_ms": train, "move_ms_total": move,
                    "move_ms_per_move": move / max(len(order) - 1, 1), "ms_per_position": (train + move) / len(order),
                    "ms_per_tile": (train + move) / (g * g), "status": ctx.sync_status(sw.tr.state),
                    "batches": "device (crops, ray pool, Philox draws)" if args.device_batches else "host",
                    "final_loss": st["loss"]})
        del sw
        torch.cuda.empty_cache()
    print(json.dumps({"workload": args.workload, "sweeps": res}), flush=True)


if __name__ == "__main__":
    _main()
