"""The snake sweep of a tile grid (oracle, FP64).  Test infrastructure only.

Sec. 4.4: a 2 x 2 window of tiles slides over the grid in snake order --
along a row of window positions, then one row up and back the other way --
so that every move keeps two tiles and exchanges the other two.  Only the
window's four tiles train at a position; each tile keeps its own optimiser
state across positions (one Adam optimiser per tile, no reset), and the
colour network is shared by all tiles.

Each tile's state is a dict of FP64 arrays (its slot block of the flat
layout: table, W1, W2, W3), Adam m and v, and its step count.  A window
position trains the flat vector [tile(0,0) | tile(1,0) | tile(0,1) |
tile(1,1) | colour] with step.train_step.
"""
import numpy as np

from . import step as S


def snake_positions(gx, gy):
    """Lower-left tiles (ix, iy) of the window positions, in visiting order."""
    order = []
    for iy in range(gy - 1):
        xs = range(gx - 1) if iy % 2 == 0 else range(gx - 2, -1, -1)
        order.extend((ix, iy) for ix in xs)
    return order


def window_tiles(pos):
    """Grid tiles of the window at pos, in window order (ix + 2 iy)."""
    return [(pos[0] + dx, pos[1] + dy) for dy in (0, 1) for dx in (0, 1)]


def init_states(cfg, tile_flat, colour_flat, grid):
    """Per-tile states from one tile's initial block (copied) and the colour block."""
    n = cfg.tile_params()
    tiles = {}
    for iy in range(grid[1]):
        for ix in range(grid[0]):
            t = tile_flat[(iy * grid[0] + ix) % len(tile_flat)]
            tiles[(ix, iy)] = {"p": np.array(t, np.float64), "m": np.zeros(n), "v": np.zeros(n), "steps": 0}
    nc = cfg.col_params() * cfg.n_colour_blocks()
    colour = {"p": np.array(colour_flat, np.float64), "m": np.zeros(nc), "v": np.zeros(nc), "steps": 0}
    return tiles, colour


def run(cfg, tiles, colour, grid, iters, cameras, win_at, batch_at, targets, seed, lr=None):
    """Sweep the grid: at every position, `iters` steps on the window's tiles.
    win_at(pos) -> Window, batch_at(pos, i) -> packed pixels; lr: Adam
    learning rate (default I-NGP's).  Returns the per-step rendered rgb (list
    of arrays) and updates tiles / colour in place."""
    outs = []
    n = cfg.tile_params()
    it = 0
    for pos in snake_positions(*grid):
        keys = window_tiles(pos)
        for i in range(iters):
            flat = np.concatenate([tiles[k]["p"] for k in keys] + [colour["p"]])
            m = np.concatenate([tiles[k]["m"] for k in keys] + [colour["m"]])
            v = np.concatenate([tiles[k]["v"] for k in keys] + [colour["v"]])
            steps = [tiles[k]["steps"] for k in keys] + [colour["steps"]]
            res = S.train_step(cfg, flat, m, v, steps, cameras, win_at(pos), batch_at(pos, i), targets, seed, it,
                               lr=lr)
            for j, k in enumerate(keys):
                sl = slice(j * n, (j + 1) * n)
                tiles[k]["p"], tiles[k]["m"], tiles[k]["v"] = res.params[sl], res.m[sl], res.v[sl]
                tiles[k]["steps"] = res.extra["steps"][j]
            colour["p"], colour["m"], colour["v"] = res.params[4 * n:], res.m[4 * n:], res.v[4 * n:]
            colour["steps"] = res.extra["steps"][4]
            outs.append(res.rgb)
            it += 1
    return outs
