"""Multiresolution hash-grid encoding (oracle, FP64).  Test infrastructure only.

Paper basis: Sec. 4.1 - each tile's NeRF queries multiresolution feature
vectors (the NGP representation of Mueller et al. 2022) at the sample's
coordinates in [0, 1]^3 of its tile.  The paper gives no formulas; this
restates NGP's encoding:

* growth factor b = exp((ln N_max - ln N_min) / (L - 1)), level resolution
  N_l = floor(N_min * b^l)  (reading: + 1e-6 inside the floor, so that the
  last level is N_max and not N_max - 1 when b^l rounds just below);
* vertices 0..N_l per axis; a level is dense when (N_l + 1)^3 <= T and then
  vertex (x, y, z) has index x + y (N_l + 1) + z (N_l + 1)^2; otherwise the
  index is (x * 1 xor y * 2654435761 xor z * 805459861) mod T, in uint32
  arithmetic (NGP's spatial hash);
* level size min(T, (N_l + 1)^3) rounded up to a multiple of 8 entries
  (reading), levels stored one after another, F features per entry;
* cell: g = x * N_l in binary32, i = min(floor(g), N_l - 1), frac = g - i
  (exact in binary32) -- the binary32 step decides the cell and must match
  the library bit for bit;
* trilinear interpolation of the 8 corner features with weights
  prod(frac or 1 - frac) in FP64; output = concatenation of the L levels'
  F-vectors, level-major.

Reading: NGP's own implementation offsets the grid by half a cell
(scale N - 1, +0.5); this restatement uses the plain g = x N_l above.
"""
from dataclasses import dataclass
import math
import numpy as np

PRIME_Y = np.uint32(2654435761)
PRIME_Z = np.uint32(805459861)


@dataclass
class GridLayout:
    L: int
    F: int
    T: int
    res: np.ndarray       # (L,) int N_l
    dense: np.ndarray     # (L,) bool
    size: np.ndarray      # (L,) int entries per level (rounded up to 8)
    offset: np.ndarray    # (L,) int first entry of the level
    n_entries: int

    @property
    def n_params(self):
        return self.n_entries * self.F


def layout(L, F, log2_T, n_min, n_max):
    T = 1 << log2_T
    if L > 1:
        b = math.exp((math.log(n_max) - math.log(n_min)) / (L - 1))
    else:
        b = 1.0
    res = np.array([int(math.floor(n_min * b ** l + 1e-6)) for l in range(L)], np.int64)
    n_vert = (res + 1) ** 3
    dense = n_vert <= T
    size = np.minimum(n_vert, T)
    size = (size + 7) // 8 * 8
    offset = np.zeros(L, np.int64)
    offset[1:] = np.cumsum(size)[:-1]
    return GridLayout(L, F, T, res, dense, size, offset, int(size.sum()))


def cells(xyz_f32, N):
    """Binary32 cell decision: g = x * N, i = min(floor(g), N - 1), frac = g - i.
    Returns int64 i (S, 3) and float32 frac (S, 3)."""
    g = (xyz_f32.astype(np.float32) * np.float32(N)).astype(np.float32)
    i = np.minimum(np.floor(g).astype(np.int64), N - 1)
    frac = (g - i.astype(np.float32)).astype(np.float32)
    return i, frac


def corner_index(ix, iy, iz, N, dense, T):
    """Entry index (within its level) of vertex (ix, iy, iz); uint32 arithmetic."""
    ix = ix.astype(np.uint64)
    iy = iy.astype(np.uint64)
    iz = iz.astype(np.uint64)
    if dense:
        n1 = np.uint64(N + 1)
        return (ix + iy * n1 + iz * n1 * n1).astype(np.int64)
    m32 = np.uint64(0xFFFFFFFF)
    h = (ix & m32) ^ ((iy * np.uint64(PRIME_Y)) & m32) ^ ((iz * np.uint64(PRIME_Z)) & m32)
    return (h & np.uint64(T - 1)).astype(np.int64)


def corners(xyz_f32, lay, level):
    """For one level: entry indices (S, 8) (global, within the tile's table) and
    FP64 trilinear weights (S, 8).  Corner c has offsets (c & 1, c >> 1 & 1, c >> 2 & 1)."""
    N = int(lay.res[level])
    i, frac = cells(xyz_f32, N)
    f = frac.astype(np.float64)
    idx = np.zeros((xyz_f32.shape[0], 8), np.int64)
    w = np.zeros((xyz_f32.shape[0], 8), np.float64)
    for c in range(8):
        b = [(c >> a) & 1 for a in range(3)]
        idx[:, c] = lay.offset[level] + corner_index(i[:, 0] + b[0], i[:, 1] + b[1], i[:, 2] + b[2], N,
                                                     bool(lay.dense[level]), lay.T)
        wc = np.ones(xyz_f32.shape[0])
        for a in range(3):
            wc = wc * (f[:, a] if b[a] else 1.0 - f[:, a])
        w[:, c] = wc
    return idx, w


def encode(xyz_f32, table, lay):
    """Features (S, L*F) float64 of points xyz (S, 3) float32 in [0, 1]^3, for a
    table (n_entries, F)."""
    S = xyz_f32.shape[0]
    out = np.zeros((S, lay.L * lay.F))
    tab = np.asarray(table, np.float64)
    for l in range(lay.L):
        idx, w = corners(xyz_f32, lay, l)
        for c in range(8):
            out[:, l * lay.F:(l + 1) * lay.F] += w[:, c:c + 1] * tab[idx[:, c]]
    return out


def encode_backward(xyz_f32, dfeat, lay):
    """Gradient of sum(dfeat * encode(xyz)) w.r.t. the table: (n_entries, F),
    contributions to the same entry (colliding vertices) added."""
    grad = np.zeros((lay.n_entries, lay.F))
    for l in range(lay.L):
        idx, w = corners(xyz_f32, lay, l)
        for c in range(8):
            np.add.at(grad, idx[:, c], w[:, c:c + 1] * dfeat[:, l * lay.F:(l + 1) * lay.F])
    return grad
