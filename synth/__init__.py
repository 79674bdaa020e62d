"""Seeded synthetic inputs for the Snake-NeRF training step.

This module is shared by the oracle, the tests and the benchmark.  It holds
none of the method's arithmetic: it only draws numbers (scene parameters,
camera coefficients, pixel batches, smooth colour images) from seeded numpy
generators.  Evaluating a camera, clipping rays, encoding, rendering and
everything else the method computes lives separately in ``oracle/`` (CPU,
FP64) and in the CUDA library.

The paper trains on the DFC2019 WorldView-3 JAX scenes (Sec. 5.1), which are
not available; these generators stand in for them with satellite-like
geometry: a few to a few dozen pushbroom views at 5-40 degrees off nadir,
a heightfield scene whose relief is small next to its horizontal extent, and
image crops of the views around each 3D tile (Sec. 4.3).
"""
from dataclasses import dataclass, field
import math
import numpy as np

CAM_AFFINE = 0
CAM_RPC3 = 1

# Cubic monomials of the normalised image/height coordinates (c, r, h), in the
# order the localisation polynomials use (RPC00B order with (L, P, H) read as
# (c, r, h)).  Each entry lists the factors of the monomial.
RPC_MONOMIALS = (
    (), ("c",), ("r",), ("h",), ("c", "r"), ("c", "h"), ("r", "h"), ("c", "c"), ("r", "r"),
    ("h", "h"), ("c", "r", "h"), ("c", "c", "c"), ("c", "r", "r"), ("c", "h", "h"),
    ("c", "c", "r"), ("r", "r", "r"), ("r", "h", "h"), ("c", "c", "h"), ("r", "r", "h"),
    ("h", "h", "h"),
)


@dataclass
class Camera:
    """One view.  kind CAM_AFFINE: x = a0 + a1 c + a2 r + a3 h, y = b0 + b1 c + b2 r + b3 h.
    kind CAM_RPC3: normalised coordinates (v - off) / scale for (r, c, h), and
    x = x_off + x_scale * Nx/Dx, y = y_off + y_scale * Ny/Dy with cubic Nx, Dx, Ny, Dy
    (coef rows 0..3, RPC_MONOMIALS order).  (r, c) are pixel coordinates of the
    full image; the pixel centre of integer pixel (row, col) is (row + 0.5, col + 0.5).
    The crop (r0, c0, h, w) is the part of the image resident for training."""
    kind: int
    width: int
    height: int
    a: np.ndarray = field(default_factory=lambda: np.zeros(4))
    b: np.ndarray = field(default_factory=lambda: np.zeros(4))
    off: np.ndarray = field(default_factory=lambda: np.zeros(5))    # r, c, h, x, y
    scale: np.ndarray = field(default_factory=lambda: np.ones(5))   # r, c, h, x, y
    coef: np.ndarray = field(default_factory=lambda: np.zeros((4, 20)))
    crop: tuple = (0, 0, 0, 0)                                       # r0, c0, h, w
    off_nadir_deg: float = 0.0
    azimuth_deg: float = 0.0


@dataclass
class Window:
    """A window of nx x ny loaded 3D tiles (Sec. 4.2, 4.4).  Boxes are in scene
    metres; tiles share z_min / z_max.  `slot[iy * nx + ix]` is the parameter slot
    of tile (ix, iy)."""
    origin: np.ndarray          # (x0, y0, z_min) of the window
    tile_size: np.ndarray       # (Wt, Ht, z_max - z_min)
    nx: int
    ny: int
    scene_lo: np.ndarray
    scene_hi: np.ndarray
    slot: tuple = (0, 1, 2, 3)


@dataclass
class Heightfield:
    """z(x, y) = z_base + sum_i a_i sin(2 pi (kx_i x + ky_i y) + phi_i)."""
    z_base: float
    amp: np.ndarray
    k: np.ndarray      # (n, 2) cycles per metre
    phase: np.ndarray
    albedo: np.ndarray  # (32, 32, 3) colour noise over the scene's xy box
    lo: np.ndarray
    hi: np.ndarray
    sun: np.ndarray


def heightfield(seed, lo, hi, n_sin=8, amplitude=20.0, min_wavelength=24.0):
    """Seeded sum-of-sinusoids heightfield with total amplitude `amplitude`
    metres inside the scene box [lo, hi] and a 32x32 colour-noise albedo."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    w = rng.uniform(0.2, 1.0, n_sin)
    amp = amplitude * w / w.sum() / 2.0   # peak-to-peak sum = amplitude
    ext = float(min(hi[0] - lo[0], hi[1] - lo[1]))
    lam = rng.uniform(min_wavelength, max(min_wavelength * 1.5, ext / 2.0), n_sin)
    ang = rng.uniform(0, 2 * np.pi, n_sin)
    k = np.stack([np.cos(ang) / lam, np.sin(ang) / lam], axis=1)
    phase = rng.uniform(0, 2 * np.pi, n_sin)
    z_base = lo[2] + 0.4 * (hi[2] - lo[2])
    albedo = rng.uniform(0.15, 0.9, (32, 32, 3))
    sun_az = rng.uniform(0, 2 * np.pi)
    sun_el = np.deg2rad(rng.uniform(40, 70))
    sun = np.array([np.cos(sun_el) * np.cos(sun_az), np.cos(sun_el) * np.sin(sun_az), np.sin(sun_el)])
    return Heightfield(z_base, amp, k, phase, albedo, lo, hi, sun)


@dataclass
class Blocks:
    """Urban-like scene: z(x, y) = H[i, j], the height of the raster cell
    (i = row along y, j = column along x) of an n x n grid over the scene's xy
    box that holds (x, y).  H is a ground level plus seeded axis-aligned
    blocks (walls are vertical, roofs flat)."""
    H: np.ndarray       # (n, n) cell heights, metres
    albedo: np.ndarray  # (32, 32, 3) colour noise over the scene's xy box
    lo: np.ndarray
    hi: np.ndarray
    sun: np.ndarray


def blocks(seed, lo, hi, n=512, coverage=0.45, height=(5.0, 60.0), side=(0.01, 0.08)):
    """Seeded blocks on an n x n raster: block heights U(height) above a ground
    level at 10 % of the box height (scaled to the box when it is lower than
    96 m), footprints U(side) x the box side per axis, drawn until about
    `coverage` of the cells are covered (overlaps take the taller block)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    zlen = hi[2] - lo[2]
    s = min(1.0, zlen / 96.0)
    ground = lo[2] + 0.1 * zlen
    H = np.full((n, n), ground)
    covered = np.zeros((n, n), bool)
    while covered.mean() < coverage:
        wx = max(1, int(rng.uniform(*side) * n))
        wy = max(1, int(rng.uniform(*side) * n))
        j0 = int(rng.integers(0, n - wx + 1))
        i0 = int(rng.integers(0, n - wy + 1))
        top = ground + s * rng.uniform(*height)
        H[i0:i0 + wy, j0:j0 + wx] = np.maximum(H[i0:i0 + wy, j0:j0 + wx], top)
        covered[i0:i0 + wy, j0:j0 + wx] = True
    albedo = rng.uniform(0.15, 0.9, (32, 32, 3))
    sun_az = rng.uniform(0, 2 * np.pi)
    sun_el = np.deg2rad(rng.uniform(40, 70))
    sun = np.array([np.cos(sun_el) * np.cos(sun_az), np.cos(sun_el) * np.sin(sun_az), np.sin(sun_el)])
    return Blocks(H, albedo, lo, hi, sun)


def pushbroom_cameras(seed, n_views, width, height, lo, hi, off_nadir=(5.0, 30.0),
                      kind=CAM_AFFINE, rpc_perturb=1e-3, footprint=1.0):
    """Seeded satellite-like views of the scene box [lo, hi].

    Each view looks at the box centre from off-nadir angle theta ~ U(off_nadir)
    and azimuth ~ U[0, 360); its image is rotated by a random angle and its
    footprint at mid-height spans `footprint` times the box's larger horizontal
    side.  The affine localisation coefficients are written down from that
    geometry.  For CAM_RPC3 the same affine map is re-expressed in normalised
    coordinates (numerators linear, denominators 1) and then perturbed with
    seeded small quadratic and cubic terms of relative size `rpc_perturb`."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    cx, cy = (lo[0] + hi[0]) / 2, (lo[1] + hi[1]) / 2
    h_ref = (lo[2] + hi[2]) / 2
    ext = max(hi[0] - lo[0], hi[1] - lo[1]) * footprint
    gsd = ext / max(width, height)
    cams = []
    for _ in range(n_views):
        theta = np.deg2rad(rng.uniform(*off_nadir))
        phi = rng.uniform(0, 2 * np.pi)
        psi = rng.uniform(0, 2 * np.pi)
        tx, ty = -np.tan(theta) * np.cos(phi), -np.tan(theta) * np.sin(phi)
        a1, a2 = gsd * np.cos(psi), -gsd * np.sin(psi)
        b1, b2 = gsd * np.sin(psi), gsd * np.cos(psi)
        a0 = cx - (a1 * width / 2 + a2 * height / 2) - tx * h_ref
        b0 = cy - (b1 * width / 2 + b2 * height / 2) - ty * h_ref
        cam = Camera(kind, width, height, a=np.array([a0, a1, a2, tx]), b=np.array([b0, b1, b2, ty]),
                     crop=(0, 0, height, width), off_nadir_deg=float(np.rad2deg(theta)),
                     azimuth_deg=float(np.rad2deg(phi)))
        if kind == CAM_RPC3:
            off = np.array([height / 2, width / 2, h_ref, cx, cy])
            scale = np.array([height / 2, width / 2, (hi[2] - lo[2]) / 2, ext / 2, ext / 2])
            coef = np.zeros((4, 20))
            # x = x_off + x_scale * (n0 + n_c cn + n_r rn + n_h hn)
            for row, (q0, qc, qr, qh, o_xy, s_xy) in enumerate(
                    [(a0, a1, a2, tx, off[3], scale[3]), (b0, b1, b2, ty, off[4], scale[4])]):
                num = np.zeros(20)
                num[0] = (q0 + qc * off[1] + qr * off[0] + qh * off[2] - o_xy) / s_xy
                num[1] = qc * scale[1] / s_xy
                num[2] = qr * scale[0] / s_xy
                num[3] = qh * scale[2] / s_xy
                num[4:] = rng.uniform(-rpc_perturb, rpc_perturb, 16)
                den = np.zeros(20)
                den[0] = 1.0
                den[1:] = rng.uniform(-rpc_perturb, rpc_perturb, 19) * 0.5
                coef[2 * row] = num
                coef[2 * row + 1] = den
            cam.off, cam.scale, cam.coef = off, scale, coef
        cams.append(cam)
    return cams


def rpc_as_affine(cam):
    """The RPC3 form of an affine camera with no perturbation (for tests):
    same normalisation as pushbroom_cameras, numerators linear, denominators 1."""
    c = Camera(CAM_RPC3, cam.width, cam.height, a=cam.a.copy(), b=cam.b.copy(), crop=cam.crop)
    c.off = np.array([cam.height / 2, cam.width / 2, 0.0, 0.0, 0.0])
    c.scale = np.array([cam.height / 2, cam.width / 2, 1.0, 1.0, 1.0])
    coef = np.zeros((4, 20))
    for row, q in enumerate([cam.a, cam.b]):
        coef[2 * row, 0] = q[0] + q[1] * c.off[1] + q[2] * c.off[0]
        coef[2 * row, 1] = q[1] * c.scale[1]
        coef[2 * row, 2] = q[2] * c.scale[0]
        coef[2 * row, 3] = q[3]
        coef[2 * row + 1, 0] = 1.0
    c.coef = coef
    return c


def pack_pixel(view, row, col):
    """Pixel id: view in bits 24..31, row in 12..23, col in 0..11 (all < 4096 / 256)."""
    view = np.asarray(view, np.uint32)
    row = np.asarray(row, np.uint32)
    col = np.asarray(col, np.uint32)
    return (view << np.uint32(24)) | (row << np.uint32(12)) | col


def unpack_pixel(pix):
    pix = np.asarray(pix, np.uint32)
    return (pix >> np.uint32(24)).astype(np.int64), ((pix >> np.uint32(12)) & np.uint32(0xFFF)).astype(np.int64), \
        (pix & np.uint32(0xFFF)).astype(np.int64)


def random_pixels(seed, n_rays, cameras, views=None):
    """Uniform random pixels of the cameras' crops (the random ray batch of Sec. 4.4)."""
    rng = np.random.default_rng(seed)
    views = np.arange(len(cameras)) if views is None else np.asarray(views)
    v = views[rng.integers(0, len(views), n_rays)]
    r = np.empty(n_rays, np.int64)
    c = np.empty(n_rays, np.int64)
    for vi in np.unique(v):
        m = v == vi
        r0, c0, h, w = cameras[vi].crop
        r[m] = r0 + rng.integers(0, h, m.sum())
        c[m] = c0 + rng.integers(0, w, m.sum())
    return pack_pixel(v, r, c)


def smooth_images(seed, n_views, height, width, grid=32):
    """Seeded smooth colour images (bilinear upsampling of grid x grid noise),
    float32 (n_views, height, width, 3) in [0.1, 0.9]."""
    rng = np.random.default_rng(seed)
    out = np.empty((n_views, height, width, 3), np.float32)
    ys = np.linspace(0, grid - 1, height)
    xs = np.linspace(0, grid - 1, width)
    y0 = np.minimum(np.floor(ys).astype(int), grid - 2)
    x0 = np.minimum(np.floor(xs).astype(int), grid - 2)
    fy = (ys - y0)[:, None, None]
    fx = (xs - x0)[None, :, None]
    for v in range(n_views):
        g = rng.uniform(0.1, 0.9, (grid, grid, 3))
        img = (g[y0][:, x0] * (1 - fy) * (1 - fx) + g[y0 + 1][:, x0] * fy * (1 - fx)
               + g[y0][:, x0 + 1] * (1 - fy) * fx + g[y0 + 1][:, x0 + 1] * fy * fx)
        out[v] = img.astype(np.float32)
    return out


def dirichlet_mix(seed, n_rays, n_tiles=4, alpha=0.5):
    """Per-tile ray counts n ~ Multinomial(n_rays, p), p ~ Dirichlet(alpha 1_n)."""
    rng = np.random.default_rng(seed)
    p = rng.dirichlet(alpha * np.ones(n_tiles))
    return rng.multinomial(n_rays, p), p


def glorot_bound(fan_in, fan_out):
    return math.sqrt(6.0 / (fan_in + fan_out))
