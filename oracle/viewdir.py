"""View-direction encoding of the colour network's input (oracle, FP64).
Test infrastructure only.

The variant of the colour network with a view-direction input follows
Instant-NGP's direction encoding (Mueller et al. 2022): the real spherical
harmonics of degrees 0..3 (16 functions) of the ray's unit direction d =
(x, y, z), appended to the 16-d density embedding.  Here they are evaluated
from their definition: Y_l^m = sqrt(2) K_l^|m| P_l^|m|(z) cos(m phi) for
m > 0, K_l^0 P_l(z) for m = 0 and sqrt(2) K_l^|m| P_l^|m|(z) sin(|m| phi)
for m < 0, with K_l^m = sqrt((2l + 1) / (4 pi) (l - m)! / (l + m)!), P_l^m the
associated Legendre functions without the Condon-Shortley phase, cos theta = z
and phi the azimuth of (x, y) -- a real orthonormal basis on the sphere, in
the order (l, m) = (0, 0), (1, -1), (1, 0), (1, 1), (2, -2), ..., (3, 3), each
multiplied by the sign (-1)^m for m odd as in the usual graphics tables (the
basis stays orthonormal; the sign only fixes a convention both sides share).
"""
import math

import numpy as np

N_SH = 16


def _assoc_legendre(l, m, z):
    """P_l^m(z) for m >= 0 without the Condon-Shortley phase (standard recurrences)."""
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    pmm = np.ones_like(z)
    for k in range(1, m + 1):
        pmm = pmm * (2 * k - 1) * s
    if l == m:
        return pmm
    pm1 = z * (2 * m + 1) * pmm
    if l == m + 1:
        return pm1
    for ll in range(m + 2, l + 1):
        pll = (z * (2 * ll - 1) * pm1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pm1 = pm1, pll
    return pm1


def sh16(d):
    """(S, 16) real spherical harmonics of unit directions d (S, 3)."""
    d = np.asarray(d, np.float64)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    phi = np.arctan2(y, x)
    out = []
    for l in range(4):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            P = _assoc_legendre(l, am, z)
            if m > 0:
                v = math.sqrt(2.0) * K * P * np.cos(am * phi)
            elif m < 0:
                v = math.sqrt(2.0) * K * P * np.sin(am * phi)
            else:
                v = K * P
            out.append(v * (-1.0 if am % 2 == 1 else 1.0))
    return np.stack(out, 1)
