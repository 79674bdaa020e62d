"""Pins of the oracle's E4M3 quantiser (oracle/quant.py) against what the
format fixes: its largest and smallest values, round-to-nearest-even ties,
saturation, the code <-> value bijection, and PyTorch's float8_e4m3fn cast (a
library conversion of the same format) wherever that cast does not overflow."""
import numpy as np
import pytest

from oracle import quant as Q


def test_known_codes_and_values():
    # 448 = 1.75 x 2^8 is the largest finite value: exponent field 15, mantissa 6
    assert Q.e4m3_encode([448.0])[0] == 0x7E
    assert Q.e4m3_decode([0x7E])[0] == 448.0
    # smallest subnormal 2^-9, smallest normal 2^-6, one
    assert Q.e4m3_encode([2.0 ** -9])[0] == 0x01
    assert Q.e4m3_encode([2.0 ** -6])[0] == 0x08
    assert Q.e4m3_encode([1.0])[0] == 0x38
    assert Q.e4m3_encode([-2.0])[0] == 0xC0
    assert np.isnan(Q.e4m3_decode([0x7F])[0]) and np.isnan(Q.e4m3_decode([0xFF])[0])


def test_ties_go_to_even_mantissa():
    # between 1 (mantissa 0) and 1.125 (mantissa 1): 1.0625 -> 1
    assert Q.e4m3_round([1.0625])[0] == 1.0
    # between 1.125 (1) and 1.25 (2): 1.1875 -> 1.25
    assert Q.e4m3_round([1.1875])[0] == 1.25
    # subnormal ties: 2^-10 (between 0 and 2^-9) -> 0; 3 x 2^-10 (between 2^-9 and 2^-8) -> 2^-8
    assert Q.e4m3_round([2.0 ** -10])[0] == 0.0
    assert Q.e4m3_round([3 * 2.0 ** -10])[0] == 2.0 ** -8
    # just off the tie rounds to the nearer value
    assert Q.e4m3_round([1.0625 + 1e-12])[0] == 1.125


def test_saturation_and_signs():
    assert Q.e4m3_round([1e9, -1e9, 463.9, 464.0, 500.0]).tolist() == [448.0, -448.0, 448.0, 448.0, 448.0]
    assert np.signbit(Q.e4m3_round([-0.0])[0])
    assert Q.e4m3_encode([-0.0])[0] == 0x80


def test_every_code_round_trips():
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], np.uint8)
    vals = Q.e4m3_decode(codes)
    assert np.array_equal(Q.e4m3_encode(vals), codes)
    assert np.array_equal(Q.e4m3_round(vals), vals)
    pos = np.sort(vals[vals > 0])
    assert len(pos) == 126 and pos[0] == 2.0 ** -9 and pos[-1] == 448.0


def test_matches_torch_float8_cast_in_range():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.normal(0, 1, 20000), rng.normal(0, 100, 20000), rng.uniform(-2.0 ** -6, 2.0 ** -6, 20000),
        np.ldexp(rng.uniform(1, 2, 20000), rng.integers(-12, 9, 20000)) * rng.choice([-1, 1], 20000)])
    # every tie between adjacent finite values as well
    vals = np.sort(Q.e4m3_decode(np.arange(0, 0x7F, dtype=np.uint8)))
    ties = 0.5 * (vals[1:] + vals[:-1])
    x = np.concatenate([x, ties, -ties]).astype(np.float32).astype(np.float64)
    x = x[np.abs(x) < 464.0]  # the library cast gives NaN from 464 on; ours saturates
    lib = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(Q.e4m3_encode(x), lib)


def test_round_is_monotone_and_within_half_a_step():
    x = np.sort(np.random.default_rng(1).uniform(-500, 500, 100000))
    r = Q.e4m3_round(x)
    assert np.all(np.diff(r) >= 0)
    a = np.abs(x)
    inside = a <= 448
    _, E = np.frexp(a)
    step = np.ldexp(1.0, np.maximum(E - 1, -6) - 3)
    assert np.all(np.abs(r - x)[inside] <= 0.5 * step[inside])


def test_binary32_features_match_the_fp64_encoding():
    """The binary32 evaluation used for the codes' decisions differs from the
    FP64 encoding by binary32 rounding only (a dropped corner or a swapped
    weight factor would not)."""
    from oracle import hashgrid
    lay = hashgrid.layout(4, 2, 11, 4, 48)
    rng = np.random.default_rng(2)
    tab = rng.uniform(-1, 1, (lay.n_entries, 2)).astype(np.float16).astype(np.float64)
    xyz = rng.random((3000, 3)).astype(np.float32)
    f64 = hashgrid.encode(xyz, tab, lay)
    f32 = Q.encode_binary32(xyz, tab, lay)
    assert np.max(np.abs(f32 - f64)) <= 16 * 2.0 ** -24 * np.max(np.abs(tab))
    s = Q.slot_scale_binary32(f32)
    assert s.dtype == np.float32 and abs(float(s) - np.max(np.abs(f32)) / 448.0) <= 2.0 ** -24 * float(s)


def test_quantise_uses_amax_over_448():
    f = np.array([[0.5, -2.0], [1.0, 0.25]])
    s = Q.slot_scale(f)
    assert s == 2.0 / 448.0
    q = Q.quantise(f, s)
    assert q[0, 1] == -2.0                      # the amax maps to 448 exactly
    assert np.all(np.abs(q - f) <= np.abs(f) * 2.0 ** -4 + s * 2.0 ** -10)
    assert Q.slot_scale(np.zeros((3, 2))) == 1.0


# ---- the quantised first layer inside the oracle's training step ----------

def _fp8_setup(n_rays=24, hidden=16, seed=0):
    from synth import workloads as W
    from oracle import step as OS, targets as OT
    w = W.get("tiny_window_fp8", n_rays=n_rays, hidden=hidden)
    cams = W.cameras(w)
    tg = OT.render_targets(W.scene(w), cams)
    cfg = OS.ModelConfig(L=w.L, F=w.F, log2_T=w.log2_T, n_min=w.n_min, n_max=w.n_max, hidden=w.hidden,
                         geo_out=w.geo_out, colour=w.colour, shared_colour=w.shared_colour, n_slots=w.n_slots,
                         K_ray=w.K_ray, K_min=w.K_min, K_max=w.K_max, first_layer="e4m3")
    lay = cfg.grid()
    flat = W.init_params(lay.n_params, cfg.geo_shapes(), cfg.col_shapes(), cfg.n_slots, cfg.n_colour_blocks(),
                         seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    for a, b, mlp_a in OS.group_ranges(cfg)[:cfg.n_slots]:
        flat[a:mlp_a] = rng.uniform(-0.5, 0.5, mlp_a - a)
    pix = W.batch(w, cams, seed + 11)
    return w, cams, tg, cfg, flat, pix


def test_e4m3_step_mlp_gradient_matches_central_differences():
    """The quantiser acts before the first layer's weights, so the MLP weight
    gradients of the quantised network are exact derivatives (central
    differences, rel 1e-6)."""
    from oracle import step as OS, render
    w, cams, tg, cfg, flat, pix = _fp8_setup()
    n = len(flat)
    res = OS.train_step(cfg, flat, np.zeros(n), np.zeros(n), [0] * cfg.n_optimisers(), cams, w.window(), pix,
                        tg, 5, 9)

    def loss(f):
        o, d, seg, smp = OS.sample_rays(cfg, cams, w.window(), pix, 5, 9, False)
        sigma, rgb_s, _ = OS.field_forward(cfg, f, smp)
        rgb, _, _, _, _ = render.composite(sigma, rgb_s, smp.t.astype(np.float64), smp.dt.astype(np.float64),
                                           seg.ray_off)
        return render.mse_loss(rgb, OS.gather_targets(cams, pix, tg), seg.ray_ok)[0]

    rng = np.random.default_rng(3)
    picks = []
    for a, b, mlp_a in OS.group_ranges(cfg):
        picks += list(rng.integers(mlp_a, b, 6))
    for p in picks:
        h = 1e-6 * max(1.0, abs(flat[p]))
        fp_, fm_ = flat.copy(), flat.copy()
        fp_[p] += h
        fm_[p] -= h
        fd = (loss(fp_) - loss(fm_)) / (2 * h)
        assert abs(fd - res.grad[p]) <= 1e-6 * abs(fd) + 1e-10, (p, fd, res.grad[p])


def test_e4m3_step_equals_f16_step_when_features_are_representable():
    """Tables constant per level with values A 2^-j: every feature is A 2^-j
    (the trilinear weights sum to one, up to binary32 rounding), amax / 448
    divides it into 448 2^-j, an E4M3 value, so the codes are exact and the
    straight-through gradient is the true one: both steps agree up to the
    binary32 rounding of the features, the amax and the scale."""
    import dataclasses
    from oracle import step as OS
    w, cams, tg, cfg, flat, pix = _fp8_setup()
    lay = cfg.grid()
    for si, (a, b, mlp_a) in enumerate(OS.group_ranges(cfg)[:cfg.n_slots]):
        tab = flat[a:mlp_a].reshape(lay.n_entries, cfg.F)
        for l in range(cfg.L):
            o, sz = int(lay.offset[l]), int(lay.size[l])
            tab[o:o + sz, 0] = 0.75 * 2.0 ** -(l % 4)
            tab[o:o + sz, 1] = -0.75 * 2.0 ** -((l + 1 + si) % 5)
    n = len(flat)
    args = (np.zeros(n), np.zeros(n), [0] * cfg.n_optimisers(), cams, w.window(), pix, tg, 5, 9)
    q = OS.train_step(cfg, flat, *args)
    f = OS.train_step(dataclasses.replace(cfg, first_layer="f16"), flat, *args)
    # the codes are exact; scale x value carries the binary32 rounding of the amax and the scale
    assert abs(q.loss - f.loss) <= 1e-6 * abs(f.loss)
    assert np.allclose(q.rgb, f.rgb, rtol=1e-6, atol=1e-9)
    assert np.linalg.norm(q.grad - f.grad) <= 1e-5 * np.linalg.norm(f.grad)
