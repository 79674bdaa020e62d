"""Pins of the oracle's volume rendering (NeRF Eq. 3 as used in Sec. 4.5), the
colour loss, its backward, and Adam (Sec. 4.6): closed forms, invariants, the
segment-wise (NeRF-XL) aggregation and finite differences (CPU only)."""
import numpy as np
import pytest

from oracle import render, adam


def _rays(rng, n_rays, kmin=1, kmax=40):
    counts = rng.integers(kmin, kmax + 1, n_rays)
    off = np.zeros(n_rays + 1, np.int64)
    off[1:] = np.cumsum(counts)
    S = off[-1]
    sigma = rng.gamma(1.0, 0.3, S)
    rgb = rng.uniform(0, 1, (S, 3))
    dt = rng.uniform(0.05, 1.5, S)
    t = np.zeros(S)
    for r in range(n_rays):
        a, b = off[r], off[r + 1]
        t[a:b] = np.cumsum(dt[a:b]) - 0.5 * dt[a:b]
    return sigma, rgb, t, dt, off


@pytest.mark.parametrize("K", [1, 2, 7, 64, 333])
def test_constant_density_slab_opacity_closed_form(K):
    """sigma constant over a slab of length L: opacity = 1 - exp(-sigma L) for any K."""
    for sig, L in [(0.01, 50.0), (0.7, 3.0), (5.0, 0.2), (2.0, 96.0)]:
        dt = np.full(K, L / K)
        t = (np.arange(K) + 0.5) * L / K
        rgb = np.tile([0.2, 0.5, 0.9], (K, 1))
        c, depth, op, tf, w = render.composite(np.full(K, sig), rgb, t, dt, np.array([0, K]))
        assert abs(op[0] - (1 - np.exp(-sig * L))) < 1e-14
        assert np.allclose(c[0], op[0] * np.array([0.2, 0.5, 0.9]), rtol=1e-13)
        assert abs(tf[0] - np.exp(-sig * L)) < 1e-15


def test_compositing_invariants():
    rng = np.random.default_rng(0)
    sigma, rgb, t, dt, off = _rays(rng, 50)
    c, depth, op, tf, w = render.composite(sigma, rgb, t, dt, off)
    for r in range(50):
        a, b = off[r], off[r + 1]
        tau = sigma[a:b] * dt[a:b]
        T = np.exp(-(np.cumsum(tau) - tau))
        assert np.all(np.diff(T) <= 0)                         # transmittance non-increasing
        assert w[a:b].sum() <= 1 + 1e-15 and np.all(w[a:b] >= 0)
        assert abs(w[a:b].sum() - (1 - tf[r])) < 1e-14          # sum w = 1 - T_final
        assert abs(op[r] - w[a:b].sum()) < 1e-15
    assert np.all(c >= 0) and np.all(c <= 1)


def test_segmentwise_aggregation_equals_flat_compositing():
    """NeRF-XL aggregation of per-segment results, C = sum_s (prod_{s'<s} T_s') C_s,
    equals compositing the concatenated samples (the segmented sampler does not
    change the rendering equation)."""
    rng = np.random.default_rng(1)
    sigma, rgb, t, dt, off = _rays(rng, 1, 30, 30)
    cuts = [0, 7, 19, 30]
    C = np.zeros(3)
    D = 0.0
    Tacc = 1.0
    for s in range(3):
        a, b = cuts[s], cuts[s + 1]
        cs, ds, _, ts, _ = render.composite(sigma[a:b], rgb[a:b], t[a:b], dt[a:b], np.array([0, b - a]))
        C += Tacc * cs[0]
        D += Tacc * ds[0]
        Tacc *= ts[0]
    cf, df, _, tf, _ = render.composite(sigma, rgb, t, dt, off)
    assert np.allclose(C, cf[0], rtol=1e-14) and abs(D - df[0]) < 1e-12 and abs(Tacc - tf[0]) < 1e-15


def test_zero_density_is_transparent_and_empty_rays_render_black():
    c, d, op, tf, w = render.composite(np.zeros(5), np.ones((5, 3)), np.arange(5.0), np.ones(5),
                                       np.array([0, 5, 5]))
    assert np.all(c == 0) and np.all(op == 0) and tf[0] == 1.0 and tf[1] == 1.0


def test_composite_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    sigma, rgb, t, dt, off = _rays(rng, 6, 3, 25)
    g = rng.normal(size=(6, 3))

    def f(s, c):
        out, _, _, _, _ = render.composite(s, c, t, dt, off)
        return np.sum(out * g)

    dsig, drgb = render.composite_backward(g, sigma, rgb, t, dt, off)
    for i in rng.choice(len(sigma), 25, replace=False):
        h = 1e-6 * max(1.0, sigma[i])
        sp = sigma.copy()
        sp[i] += h
        sm = sigma.copy()
        sm[i] -= h
        fd = (f(sp, rgb) - f(sm, rgb)) / (2 * h)
        assert abs(fd - dsig[i]) <= 1e-7 * max(1.0, abs(fd))
        for ch in range(3):
            cp = rgb.copy()
            cp[i, ch] += 1e-6
            cm = rgb.copy()
            cm[i, ch] -= 1e-6
            fd = (f(sigma, cp) - f(sigma, cm)) / 2e-6
            assert abs(fd - drgb[i, ch]) <= 1e-7 * max(1.0, abs(fd))


def test_mse_loss_and_gradient():
    rng = np.random.default_rng(3)
    pred = rng.uniform(size=(10, 3))
    gt = rng.uniform(size=(10, 3))
    ok = np.array([1, 1, 0, 1, 1, 1, 0, 1, 1, 1], np.uint8)
    loss, g = render.mse_loss(pred, gt, ok)
    m = ok.astype(bool)
    assert abs(loss - np.mean((pred[m] - gt[m]) ** 2)) < 1e-15
    assert np.all(g[~m] == 0)
    i, ch = 3, 1
    p2 = pred.copy()
    p2[i, ch] += 1e-6
    p3 = pred.copy()
    p3[i, ch] -= 1e-6
    fd = (render.mse_loss(p2, gt, ok)[0] - render.mse_loss(p3, gt, ok)[0]) / 2e-6
    assert abs(fd - g[i, ch]) < 1e-9


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient g the bias-corrected moments are m = g, v = g^2 at
    every step, so each update moves by lr * sign(g) (eps negligible)."""
    w = np.array([0.5, -1.0, 2.0, 0.0])
    g = np.array([3e-3, -7.0, 1e-5, 2.0])
    m = np.zeros(4)
    v = np.zeros(4)
    w0 = w.copy()
    for t in range(1, 6):
        w, m, v = adam.step(w, g, m, v, t)
        assert np.allclose(w, w0 - t * adam.LR * np.sign(g), rtol=0, atol=1e-10)


def test_adam_two_steps_worked_example():
    """Worked by hand: g1 = 1, g2 = -1, lr = 0.1, beta1 = 0.5, beta2 = 0.75, eps = 0:
    step 1: m = 0.5, v = 0.25, mhat = 1, vhat = 1, w = 1 - 0.1 = 0.9;
    step 2: m = 0.25 - 0.5 = -0.25, v = 0.1875 + 0.25 = 0.4375, mhat = -0.25/0.75 = -1/3,
            vhat = 0.4375/0.4375 = 1, w = 0.9 + 0.1/3."""
    w, m, v = adam.step(np.array([1.0]), np.array([1.0]), np.zeros(1), np.zeros(1), 1, lr=0.1, beta1=0.5,
                        beta2=0.75, eps=0.0)
    assert abs(w[0] - 0.9) < 1e-15
    w, m, v = adam.step(w, np.array([-1.0]), m, v, 2, lr=0.1, beta1=0.5, beta2=0.75, eps=0.0)
    assert abs(w[0] - (0.9 + 0.1 / 3)) < 1e-15


def test_adam_weight_decay_adds_to_gradient():
    w, _, _ = adam.step(np.array([2.0]), np.array([0.0]), np.zeros(1), np.zeros(1), 1, l2=1e-3)
    assert abs(w[0] - (2.0 - adam.LR)) < 1e-12       # g' = 2e-3 > 0: moves by lr
