"""Philox-4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC 2011).  Test infrastructure only.

The paper draws a random ray batch per iteration (Sec. 4.4) and random sample
positions (stratified sampling inside each segment, Sec. 4.5); it does not say
how.  Reading: a counter-based generator, so that the GPU and this oracle can
draw the same numbers independently.  Key = (seed, iteration), counter =
(index0, index1, stream, 0).

Uniform floats: u = (x >> 8) * 2^-24, exact in binary32 and binary64.

Pinned by the published known-answer vectors (tests/test_oracle_philox.py).
"""
import numpy as np

# Round multipliers and Weyl key increments of Philox-4x32 (Salmon et al. 2011).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)

STREAM_JITTER = 1


def _mulhilo(a_u64, b_u32):
    prod = a_u64 * b_u32.astype(np.uint64)
    return (prod >> np.uint64(32)).astype(np.uint32), (prod & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def philox4x32(ctr, key, rounds=10):
    """ctr: uint32 array (..., 4); key: uint32 array (..., 2) (broadcastable).
    Returns uint32 array (..., 4)."""
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    with np.errstate(over="ignore"):
        for r in range(rounds):
            if r > 0:
                k0 = (k0 + _W0).astype(np.uint32)
                k1 = (k1 + _W1).astype(np.uint32)
            hi0, lo0 = _mulhilo(_M0, c0)
            hi1, lo1 = _mulhilo(_M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack(np.broadcast_arrays(c0, c1, c2, c3), axis=-1).astype(np.uint32)


def to_unit_float(x_u32):
    """(x >> 8) * 2^-24 in [0, 1); exact in binary32 and binary64."""
    return (np.asarray(x_u32, dtype=np.uint32) >> np.uint32(8)).astype(np.float64) * (2.0 ** -24)


def jitter(seed, iteration, ray_index, sample_index):
    """Stratified-sampling jitter u for sample `sample_index` (counted along the
    whole ray, across segments) of ray `ray_index` of the batch.
    One Philox call gives four uniforms: counter = (ray, j >> 2, STREAM_JITTER, 0),
    lane j & 3.  Returns float64 values that are exact float32 numbers."""
    ray_index = np.asarray(ray_index, dtype=np.uint32)
    sample_index = np.asarray(sample_index, dtype=np.uint32)
    ray_index, sample_index = np.broadcast_arrays(ray_index, sample_index)
    ctr = np.stack([ray_index, sample_index >> np.uint32(2),
                    np.full_like(ray_index, STREAM_JITTER), np.zeros_like(ray_index)], axis=-1)
    key = np.array([seed & 0xFFFFFFFF, iteration & 0xFFFFFFFF], dtype=np.uint32)
    out = philox4x32(ctr, key)
    lane = (sample_index & np.uint32(3)).astype(np.int64)
    bits = np.take_along_axis(out, lane[..., None], axis=-1)[..., 0]
    return to_unit_float(bits)
