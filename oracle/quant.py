"""E4M3 quantisation of the first MLP layer's input (FP64).  Test
infrastructure only.

The mixed-precision stress configuration feeds the density MLP's first layer
with 8-bit floating-point activations, one scale per tensor taken from the
current batch: scale = amax / 448, code = E4M3(x / scale), and the layer sees
scale * value(code).  The first layer's input of a slot is the slot's
encoded feature tensor, so there is one scale per slot and step.

E4M3 is the OCP 8-bit floating-point format with 1 sign bit, 4 exponent bits
(bias 7) and 3 mantissa bits, no infinities, the all-ones pattern reserved for
NaN, so the largest finite magnitude is 1.75 * 2^8 = 448 and the smallest
subnormal 2^-9.  Rounding is to nearest, ties to even, and magnitudes beyond
448 saturate to 448 (the "satfinite" conversion).

The backward treats the quantiser as the identity (straight-through
estimator, Bengio et al. 2013): d(scale * value(code)) / dx = 1.

A code is an integer that floating point decides, so the oracle takes that
decision in the precision of the kernel that takes it: binary32 features
(encode_binary32), a binary32 amax and scale, a binary32 division, then the
exact E4M3 rounding.  Everything after the code (scale * value, the MLPs) is
FP64.
"""
import numpy as np

from . import hashgrid

E4M3_MAX = 448.0
E4M3_MIN_EXP = -6      # exponent of the smallest normal, 2^-6
E4M3_MANT = 3


def e4m3_round(x):
    """Nearest E4M3 value to each x (FP64), ties to even, saturating at +-448."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, E = np.frexp(a)                      # a = m 2^E, m in [0.5, 1)
    e = np.maximum(E - 1, E4M3_MIN_EXP)     # binade of a (subnormals share the lowest)
    quantum = np.ldexp(1.0, e - E4M3_MANT)  # spacing of E4M3 values in that binade
    r = np.round(a / quantum) * quantum     # a / quantum is exact; np.round is ties-to-even
    r = np.minimum(r, E4M3_MAX)
    return np.copysign(r, x)


def e4m3_encode(x):
    """uint8 codes of e4m3_round(x): sign << 7 | exponent field << 3 | mantissa."""
    r = e4m3_round(x)
    a = np.abs(r)
    sign = (np.signbit(r)).astype(np.uint8) << 7
    _, E = np.frexp(a)
    normal = a >= 2.0 ** E4M3_MIN_EXP
    e = np.where(normal, E - 1, E4M3_MIN_EXP)
    field = np.where(normal, e + 7, 0)
    frac = np.where(normal, a / np.ldexp(1.0, e) - 1.0, a / np.ldexp(1.0, E4M3_MIN_EXP))
    mant = np.rint(frac * 8).astype(np.int64)
    code = sign | (field.astype(np.uint8) << 3) | mant.astype(np.uint8)
    return np.where(a == 0, sign, code).astype(np.uint8)


def e4m3_decode(code):
    """FP64 value of uint8 codes (NaN for the two NaN patterns)."""
    c = np.asarray(code, np.uint8).astype(np.int64)
    s = np.where(c >> 7, -1.0, 1.0)
    field = (c >> 3) & 15
    mant = c & 7
    v = np.where(field == 0, mant / 8.0 * 2.0 ** E4M3_MIN_EXP, (1.0 + mant / 8.0) * np.ldexp(1.0, field - 7))
    v = np.where((field == 15) & (mant == 7), np.nan, v)
    return s * v


def _fma32(a, b, c):
    """Binary32 fused multiply-add a * b + c, rounded once: a * b (a binary32
    weight times an FP16 value, at most 35 significant bits) is exact in
    binary64, and so is the sum unless the terms lie ~18 binades apart."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def encode_binary32(xyz_f32, table, lay):
    """Features (S, L*F) as a binary32 kernel evaluates them, for the
    quantiser's decisions: per level the cell and fraction of hashgrid.cells,
    per corner c = 0..7 in order the weight w_c = product of the x, y, z
    factors (frac or 1 - frac, binary32, left to right) and f <- fma(w_c, v_c,
    f) from f = 0, v_c the table entry as binary32 (exact for FP16 tables)."""
    S = xyz_f32.shape[0]
    tab = np.asarray(table, np.float64).astype(np.float32)
    out = np.zeros((S, lay.L * lay.F), np.float32)
    one = np.float32(1.0)
    for l in range(lay.L):
        N = int(lay.res[l])
        i, fr = hashgrid.cells(xyz_f32, N)
        for c in range(8):
            b = [(c >> a) & 1 for a in range(3)]
            e = lay.offset[l] + hashgrid.corner_index(i[:, 0] + b[0], i[:, 1] + b[1], i[:, 2] + b[2], N,
                                                      bool(lay.dense[l]), lay.T)
            fac = [fr[:, a] if b[a] else (one - fr[:, a]).astype(np.float32) for a in range(3)]
            w = ((fac[0] * fac[1]).astype(np.float32) * fac[2]).astype(np.float32)
            for k in range(lay.F):
                out[:, l * lay.F + k] = _fma32(w, tab[e, k], out[:, l * lay.F + k])
    return out


def slot_scale_binary32(feat32):
    """The kernel's per-slot scale: amax / 448 with a binary32 amax and a
    binary32 division (1 for an empty or all-zero slot)."""
    a = np.float32(np.max(np.abs(feat32))) if feat32.size else np.float32(0.0)
    return np.float32(a / np.float32(E4M3_MAX)) if a > 0 else np.float32(1.0)


def quantise_binary32(feat32, scale32):
    """scale * E4M3(feat / scale) with the division in binary32 (FP64 result)."""
    x = (np.asarray(feat32, np.float32) / np.float32(scale32)).astype(np.float32)
    return float(scale32) * e4m3_round(x.astype(np.float64))


def slot_scale(feat):
    """Per-tensor scale of a slot's first-layer input: amax / 448 (1 if the
    tensor is empty or all zero)."""
    a = float(np.max(np.abs(feat))) if feat.size else 0.0
    return a / E4M3_MAX if a > 0 else 1.0


def quantise(feat, scale):
    """The first layer's input as the quantised path sees it: scale * E4M3(feat / scale)."""
    return scale * e4m3_round(np.asarray(feat, np.float64) / scale)
