"""Pins of the oracle's hash-grid encoding (NGP, Sec. 4.1) and MLPs against
closed forms, exact adjoints and finite differences (CPU only)."""
import numpy as np
import pytest

from oracle import hashgrid, mlp


def test_level_layouts_of_the_workloads():
    lay = hashgrid.layout(16, 2, 19, 16, 2048)
    assert lay.res[0] == 16 and lay.res[-1] == 2048
    assert list(np.flatnonzero(lay.dense)) == [0, 1, 2, 3, 4]    # 5 dense, 11 hashed levels
    assert np.all(lay.size[lay.dense] >= (lay.res[lay.dense] + 1) ** 3)
    assert np.all(lay.size[~lay.dense] == 1 << 19)
    assert np.all(lay.size % 8 == 0)
    assert lay.offset[0] == 0 and np.all(np.diff(lay.offset) == lay.size[:-1])
    lay1 = hashgrid.layout(8, 2, 14, 16, 256)
    assert lay1.res[-1] == 256 and lay1.dense.sum() == 2
    # geometric growth b = (N_max / N_min)^(1/(L-1)) within the floor
    b = (2048 / 16) ** (1 / 15)
    assert np.all(np.abs(lay.res - 16 * b ** np.arange(16)) < 1.0)


# NGP's spatial hash at T = 2^19, worked out by hand for a few vertices: the uint32 products
# y * 2654435761 and z * 805459861 (reduced mod 2^32), their xor with x, then the low 19 bits.
HASH_T19 = [
    # (x, y, z): y*Py mod 2^32, z*Pz mod 2^32, xor, index
    ((1, 0, 0), 0, 0, 0x00000001, 1),
    # 0x9e3779b1 & 0x7ffff = 0x779b1
    ((0, 1, 0), 2654435761, 0, 0x9E3779B1, 489905),
    # 0x30025795 & 0x7ffff = 0x25795
    ((0, 0, 1), 0, 805459861, 0x30025795, 153493),
    # 5 * 2654435761 = 13272178805 = 3 * 2^32 + 387276917; 7 * 805459861 = 5638219027 = 2^32 + 1343251731
    ((3, 5, 7), 387276917, 1343251731, 0x47050565, 329061),
    # 2048 * 805459861 = 1649581795328 = 384 * 2^32 + 314353664
    ((2047, 1, 2048), 2654435761, 314353664, 0x8C8BD64E, 251470),
    # 4001 * 2654435761 = 10620397479761 = 2472 * 2^32 + 3238324049;
    # 4002 * 805459861 = 3223450363722 = 750 * 2^32 + 2224891722
    ((4000, 4001, 4002), 3238324049, 2224891722, 0x4599CFBB, 118715),
]


@pytest.mark.parametrize("xyz,py,pz,h,index", HASH_T19)
def test_spatial_hash_known_values(xyz, py, pz, h, index):
    x, y, z = xyz
    assert x ^ py ^ pz == h and h & ((1 << 19) - 1) == index    # the table is self-consistent
    got = hashgrid.corner_index(np.array([x]), np.array([y]), np.array([z]), 0, False, 1 << 19)[0]
    assert got == index


def _trilinear_field(rng):
    c = rng.normal(size=8)

    def f(x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * x * z + c[6] * y * z
                + c[7] * x * y * z)
    return f


def test_dense_levels_reproduce_trilinear_fields_exactly():
    """Table = f(vertex / N) with f trilinear => encode(x) = f(x) at dense levels."""
    lay = hashgrid.layout(3, 2, 16, 4, 20)
    assert lay.dense.all()
    rng = np.random.default_rng(0)
    fs = [[_trilinear_field(rng) for _ in range(2)] for _ in range(3)]
    table = np.zeros((lay.n_entries, 2))
    for l in range(3):
        N = int(lay.res[l])
        v = np.arange(N + 1)
        X, Y, Z = np.meshgrid(v, v, v, indexing="ij")
        idx = lay.offset[l] + X + Y * (N + 1) + Z * (N + 1) ** 2     # x fastest
        for f in range(2):
            table[idx.ravel(), f] = fs[l][f](X.ravel() / N, Y.ravel() / N, Z.ravel() / N)
    xyz = rng.uniform(0, 1, (500, 3)).astype(np.float32)
    xyz[:5] = [[0, 0, 0], [1, 1, 1], [0.5, 0.25, 1], [1, 0, 0.75], [0.125, 1, 0]]
    out = hashgrid.encode(xyz, table, lay)
    for l in range(3):
        # the level evaluates the field at its binary32 grid coordinate g = fl(x N), i.e. at g / N
        N = int(lay.res[l])
        x64 = (xyz * np.float32(N)).astype(np.float32).astype(np.float64) / N
        assert np.max(np.abs(x64 - xyz)) < 1e-6
        for f in range(2):
            assert np.max(np.abs(out[:, 2 * l + f] - fs[l][f](x64[:, 0], x64[:, 1], x64[:, 2]))) < 1e-12


def test_hashed_levels_interpolate_the_eight_hashed_corners():
    """At a hashed level every feature is a convex combination (weights sum to 1)
    of the entries at the 8 hashed corners; a table that is 1 everywhere
    encodes to 1, and one-hot tables give the corner weights."""
    lay = hashgrid.layout(2, 2, 6, 8, 30)
    assert not lay.dense[1]
    rng = np.random.default_rng(1)
    xyz = rng.uniform(0, 1, (200, 3)).astype(np.float32)
    out = hashgrid.encode(xyz, np.ones((lay.n_entries, 2)), lay)
    assert np.allclose(out, 1.0, atol=1e-13)
    idx, w = hashgrid.corners(xyz, lay, 1)
    assert np.allclose(w.sum(1), 1.0, atol=1e-14) and np.all(w >= 0)
    assert np.all((idx >= lay.offset[1]) & (idx < lay.offset[1] + lay.size[1]))


def test_cell_decision_at_vertices_and_upper_face():
    i, frac = hashgrid.cells(np.array([[0.0, 1.0, 0.5]], np.float32), 16)
    assert list(i[0]) == [0, 15, 8] and list(frac[0]) == [0.0, 1.0, 0.0]


def test_encode_backward_is_the_exact_adjoint():
    """<encode(table), dfeat> == <table, encode_backward(dfeat)> for any table,
    colliding hashed entries included."""
    lay = hashgrid.layout(4, 2, 8, 4, 64)
    rng = np.random.default_rng(2)
    xyz = rng.uniform(0, 1, (300, 3)).astype(np.float32)
    table = rng.normal(size=(lay.n_entries, 2))
    dfeat = rng.normal(size=(300, lay.L * 2))
    lhs = np.sum(hashgrid.encode(xyz, table, lay) * dfeat)
    rhs = np.sum(table * hashgrid.encode_backward(xyz, dfeat, lay))
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def _mlp_params(rng, in_dim, hidden, G, colour):
    geo = [rng.normal(size=(hidden, in_dim)) * 0.5, rng.normal(size=(hidden, hidden)) * 0.3,
           rng.normal(size=(G, hidden)) * 0.3]
    col = [rng.normal(size=(hidden, G)) * 0.5, rng.normal(size=(hidden, hidden)) * 0.3,
           rng.normal(size=(3, hidden)) * 0.3] if colour else None
    return geo, col


def test_mlp_hand_computable_case():
    """W1 copies features, W2 the identity, W3 picks hidden unit 0 for g_0 and
    units 1..3 for g_1..3: sigma = exp(relu(x0)), rgb = sigmoid(relu(x1..3))."""
    x = np.array([[0.3, -0.2, 0.7, 1.5], [-1.0, 2.0, 0.0, -0.5]])
    W1 = np.zeros((8, 4))
    W1[:4, :4] = np.eye(4)
    W2 = np.eye(8)
    W3 = np.zeros((4, 8))
    W3[:, :4] = np.eye(4)
    sigma, rgb, _ = mlp.forward(x, [W1, W2, W3], None)
    r = np.maximum(x, 0)
    assert np.allclose(sigma, np.exp(r[:, 0]), rtol=1e-15)
    assert np.allclose(rgb, 1 / (1 + np.exp(-r[:, 1:4])), rtol=1e-15)


@pytest.mark.parametrize("colour", [False, True])
def test_mlp_backward_matches_central_differences(colour):
    rng = np.random.default_rng(4)
    G = 16 if colour else 4
    geo, col = _mlp_params(rng, 8, 12, G, colour)
    x = rng.normal(size=(40, 8))
    ds = rng.normal(size=40)
    dr = rng.normal(size=(40, 3))

    def f(geo_, col_, x_):
        s, c, _ = mlp.forward(x_, geo_, col_)
        return np.sum(ds * s) + np.sum(dr * c)

    _, _, acts = mlp.forward(x, geo, col)
    dgeo, dcol, dx = mlp.backward(ds, dr, geo, col, acts)
    mats = [("g", k) for k in range(3)] + ([("c", k) for k in range(3)] if colour else [])
    for kind, k in mats:
        W = geo[k] if kind == "g" else col[k]
        an = dgeo[k] if kind == "g" else dcol[k]
        for (a, b) in [(0, 0), (1, 2), (W.shape[0] - 1, W.shape[1] - 1), (2, 1)]:
            if a >= W.shape[0] or b >= W.shape[1]:
                continue
            h = 1e-6 * max(1.0, abs(W[a, b]))
            old = W[a, b]
            W[a, b] = old + h
            fp = f(geo, col, x)
            W[a, b] = old - h
            fm = f(geo, col, x)
            W[a, b] = old
            fd = (fp - fm) / (2 * h)
            assert abs(fd - an[a, b]) <= 1e-6 * max(1.0, abs(fd))
    for (i, j) in [(0, 0), (5, 3), (39, 7)]:
        h = 1e-6
        xp = x.copy()
        xp[i, j] += h
        xm = x.copy()
        xm[i, j] -= h
        fd = (f(geo, col, xp) - f(geo, col, xm)) / (2 * h)
        assert abs(fd - dx[i, j]) <= 1e-6 * max(1.0, abs(fd))


def test_truncated_exponential_gradient():
    """d sigma / d g_0 = exp(clamp(g_0, -15, 15)): beyond 15 the gradient stops growing."""
    W1 = np.zeros((2, 1))
    W1[0, 0] = 1.0
    W2 = np.eye(2)
    W3 = np.zeros((4, 2))
    W3[0, 0] = 1.0
    x = np.array([[3.0], [20.0]])
    _, _, acts = mlp.forward(x, [W1, W2, W3], None)
    dgeo, _, dx = mlp.backward(np.ones(2), np.zeros((2, 3)), [W1, W2, W3], None, acts)
    assert np.allclose(dx[:, 0], [np.exp(3.0), np.exp(15.0)], rtol=1e-14)


def test_view_direction_encoding_is_an_orthonormal_basis():
    """The 16 real spherical harmonics of degree <= 3 are orthonormal on the sphere:
    Gauss-Legendre in z (8 nodes) x 16 equal steps in azimuth integrate their
    products (degree <= 6) exactly."""
    from oracle import viewdir
    zn, zw = np.polynomial.legendre.leggauss(8)
    phi = np.arange(16) * (2 * np.pi / 16)
    z = np.repeat(zn, 16)
    wgt = np.repeat(zw, 16) * (2 * np.pi / 16)
    p = np.tile(phi, 8)
    s = np.sqrt(1 - z * z)
    d = np.stack([s * np.cos(p), s * np.sin(p), z], 1)
    Y = viewdir.sh16(d)
    G = (Y * wgt[:, None]).T @ Y
    assert np.allclose(G, np.eye(16), atol=1e-12)
    # degree l is odd / even under d -> -d
    Yn = viewdir.sh16(-d)
    par = np.array([1] + [-1] * 3 + [1] * 5 + [-1] * 7)
    assert np.allclose(Yn, Y * par[None, :], atol=1e-13)


def test_view_direction_encoding_closed_forms_and_addition_theorem():
    """Textbook closed forms of all 16 real harmonics (with the graphics-table
    sign (-1)^m for odd m), and the addition theorem sum_m Y_lm(d)^2 = (2l + 1) / 4 pi,
    which fixes each degree's normalisation independently of order and sign."""
    from oracle import viewdir
    rng = np.random.default_rng(3)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x, y, z = d.T
    Y = viewdir.sh16(d)
    pi = np.pi
    c1 = np.sqrt(3 / (4 * pi))
    want = {0: np.full_like(x, 0.5 / np.sqrt(pi)),
            1: -c1 * y, 2: c1 * z, 3: -c1 * x,                                   # (1, -1), (1, 0), (1, 1)
            4: 0.5 * np.sqrt(15 / pi) * x * y,                                   # (2, -2)
            6: 0.25 * np.sqrt(5 / pi) * (3 * z * z - 1),                         # (2, 0)
            8: 0.25 * np.sqrt(15 / pi) * (x * x - y * y),                        # (2, 2)
            12: 0.25 * np.sqrt(7 / pi) * (5 * z ** 3 - 3 * z),                   # (3, 0)
            10: 0.5 * np.sqrt(105 / pi) * x * y * z,                             # (3, -2)
            5: -0.5 * np.sqrt(15 / pi) * y * z, 7: -0.5 * np.sqrt(15 / pi) * x * z,  # (2, -1), (2, 1)
            9: -0.25 * np.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),         # (3, -3)
            11: -0.25 * np.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),            # (3, -1)
            13: -0.25 * np.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),            # (3, 1)
            14: 0.25 * np.sqrt(105 / pi) * z * (x * x - y * y),                  # (3, 2)
            15: -0.25 * np.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y)}        # (3, 3)
    assert sorted(want) == list(range(16))
    for j, v in want.items():
        assert np.allclose(Y[:, j], v, atol=1e-13), j
    for l in range(4):
        assert np.allclose((Y[:, l * l:(l + 1) ** 2] ** 2).sum(1), (2 * l + 1) / (4 * pi), atol=1e-13), l


def test_view_direction_colour_input_gradients_match_central_differences():
    """Colour MLP on [g | SH(d)]: the colour-weight gradients (including the direction
    columns of V1) and the embedding gradient are exact derivatives."""
    from oracle import viewdir
    rng = np.random.default_rng(4)
    S, G, H = 7, 16, 16
    feat = rng.normal(size=(S, 8))
    geo = [rng.normal(size=(H, 8)) * 0.5, rng.normal(size=(H, H)) * 0.3, rng.normal(size=(G, H)) * 0.3]
    col = [rng.normal(size=(H, G + 16)) * 0.3, rng.normal(size=(H, H)) * 0.3, rng.normal(size=(3, H)) * 0.3]
    d = rng.normal(size=(S, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    sh = viewdir.sh16(d)
    ds, dr = rng.normal(size=S), rng.normal(size=(S, 3))

    def f(cols):
        s_, r_, _ = mlp.forward(feat, geo, cols, sh)
        return float((ds * s_).sum() + (dr * r_).sum())

    _, _, acts = mlp.forward(feat, geo, col, sh)
    dgeo, dcol, dfeat = mlp.backward(ds, dr, geo, col, acts)
    h = 1e-6
    for (i, j) in [(0, 3), (5, G + 2), (9, G + 15), (2, 0)]:
        cp, cm = [c.copy() for c in col], [c.copy() for c in col]
        cp[0][i, j] += h
        cm[0][i, j] -= h
        fd = (f(cp) - f(cm)) / (2 * h)
        assert abs(fd - dcol[0][i, j]) <= 1e-6 * max(1.0, abs(fd))
    assert dfeat.shape == (S, 8)
