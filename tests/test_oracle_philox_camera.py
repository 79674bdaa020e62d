"""Pins of the oracle's RNG and camera/ray step against published vectors and
closed forms (CPU only)."""
import os
import numpy as np
import pytest

import synth
from synth import workloads as W
from oracle import philox, camera

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    out = philox.philox4x32(np.array(ctr, np.uint32), np.array(key, np.uint32))
    assert [int(x) for x in out] == expect


def test_jitter_is_exact_binary32_in_unit_interval():
    u = philox.jitter(3, 7, np.arange(100)[:, None], np.arange(50)[None, :])
    assert u.shape == (100, 50)
    assert np.all(u >= 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    # four consecutive samples share one Philox call, lanes 0..3
    raw = philox.philox4x32(np.array([5, 1, philox.STREAM_JITTER, 0], np.uint32), np.array([3, 7], np.uint32))
    assert np.array_equal(philox.jitter(3, 7, 5, np.arange(4, 8)), (raw >> 8) * 2.0 ** -24)
    # roughly uniform
    assert abs(u.mean() - 0.5) < 0.02


def test_affine_ray_direction_matches_view_geometry():
    """The synthetic view with off-nadir theta and azimuth phi has rays going
    down at angle theta from the vertical, tilted towards +phi."""
    w = W.get("tile256_fp32")
    cams = W.cameras(w)
    for vi, cam in enumerate(cams):
        pix = synth.pack_pixel([vi] * 3, [0, 40, 127], [0, 90, 127])
        o, d = camera.rays_fp64(cams, pix, np.zeros(3), 0.0, 64.0)
        th = np.deg2rad(cam.off_nadir_deg)
        ph = np.deg2rad(cam.azimuth_deg)
        expect = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), -np.cos(th)])
        assert np.allclose(d, expect[None, :], atol=1e-12)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
        assert np.allclose(o[:, 2], 64.0)


def test_affine_image_centre_sees_scene_centre():
    w = W.get("tile256_fp32")
    cams = W.cameras(w)
    for cam in cams:
        x, y = camera.localise(cam, cam.height / 2, cam.width / 2, 32.0)
        assert abs(x - 128.0) < 1e-9 and abs(y - 128.0) < 1e-9


def test_rpc_without_perturbation_reduces_to_affine():
    w = W.get("tile256_fp32")
    cams = W.cameras(w)
    rng = np.random.default_rng(0)
    r = rng.uniform(0, 128, 50)
    c = rng.uniform(0, 128, 50)
    h = rng.uniform(0, 64, 50)
    for cam in cams:
        xa, ya = camera.localise(cam, r, c, h)
        xr, yr = camera.localise(synth.rpc_as_affine(cam), r, c, h)
        assert np.max(np.abs(xa - xr)) < 1e-12 * 300 and np.max(np.abs(ya - yr)) < 1e-12 * 300
    lo, hi = np.zeros(3), np.array([256.0, 256.0, 64.0])
    rpc = synth.pushbroom_cameras(9, 4, 128, 128, lo, hi, kind=synth.CAM_RPC3, rpc_perturb=0.0)
    for cr in rpc:
        ca = synth.Camera(synth.CAM_AFFINE, cr.width, cr.height, a=cr.a, b=cr.b)
        xa, ya = camera.localise(ca, r, c, h)
        xr, yr = camera.localise(cr, r, c, h)
        assert np.max(np.abs(xa - xr)) < 1e-9 and np.max(np.abs(ya - yr)) < 1e-9


@pytest.mark.parametrize("i", range(20))
def test_rpc_monomial_convention(i):
    """Coefficient e_i on the x numerator gives x = x_off + x_scale * m_i(cn, rn, hn)
    with m_i the product of the factors the convention lists."""
    cam = synth.Camera(synth.CAM_RPC3, 100, 80)
    cam.off = np.array([40.0, 50.0, 10.0, 3.0, -2.0])
    cam.scale = np.array([40.0, 50.0, 20.0, 7.0, 5.0])
    cam.coef = np.zeros((4, 20))
    cam.coef[0, i] = 1.0
    cam.coef[1, 0] = 2.0
    cam.coef[2, 0] = 1.0
    cam.coef[3, 0] = 1.0
    r, c, h = 13.0, 77.0, 25.0
    vals = {"r": (r - 40.0) / 40.0, "c": (c - 50.0) / 50.0, "h": (h - 10.0) / 20.0}
    m = 1.0
    for f in synth.RPC_MONOMIALS[i]:
        m *= vals[f]
    x, y = camera.localise(cam, r, c, h)
    assert abs(x - (3.0 + 7.0 * m / 2.0)) < 1e-14
    assert abs(y - (-2.0 + 5.0)) < 1e-14


def test_binary32_rays_are_rounded_fp64_rays():
    w = W.get("tile512_full", n_rays=256)
    cams = W.cameras(w)
    pix = W.batch(w, cams, 1)
    o64, d64 = camera.rays_fp64(cams, pix, np.zeros(3), 0.0, 96.0)
    o, d = camera.rays(cams, pix, np.zeros(3), 0.0, 96.0)
    assert o.dtype == np.float32 and d.dtype == np.float32
    assert np.array_equal(o, o64.astype(np.float32)) and np.array_equal(d, d64.astype(np.float32))
