"""The C-ABI library loads, exports every function include/snk.h declares, its
structs match the binding's mirrors, and its host-only layout agrees with the
oracle's (CPU only: no compute call needs a GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2507_01631_b300 import build, snk
from oracle import hashgrid
from synth import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return snk.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "snk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(snk_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(snk.SIGNATURES), set(names) ^ set(snk.SIGNATURES)


def test_struct_sizes_match_the_binding(lib):
    sizes = (ctypes.c_int64 * 9)()
    assert lib.snk_abi_sizes(sizes, 9) == 9
    for s, cls in zip(sizes, snk.STRUCTS):
        assert s == ctypes.sizeof(cls), cls.__name__
    assert lib.snk_version().startswith(b"libsnk")


def test_struct_fields_match_the_binding():
    """Field names and order of every struct in include/snk.h against the binding's mirror
    (sizes alone miss two swapped or renamed fields of one type)."""
    text = re.sub(r"/\*.*?\*/|//[^\n]*", "", open(os.path.join(ROOT, "include", "snk.h")).read(), flags=re.S)
    structs = {name: body for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(snk_\w+);", text, flags=re.S)}
    for cls in snk.STRUCTS:
        cname = "snk_" + cls.__name__[3:].lower()
        assert cname in structs, cname
        fields = []
        for decl in structs[cname].split(";"):
            decl = decl.strip()
            if decl:
                fields += [re.sub(r"\[.*\]", "", v).strip().split()[-1].lstrip("*") for v in decl.split(",")]
        assert fields == [f for f, _ in cls._fields_], (cname, fields)


@pytest.mark.parametrize("name", list(W.WORKLOADS))
def test_model_layout_matches_the_oracle(lib, name):
    w = W.get(name)
    from paper_2507_01631_b300.trainer import model_from_workload
    lay = snk.layout(model_from_workload(w))
    ref = hashgrid.layout(w.L, w.F, w.log2_T, w.n_min, w.n_max)
    assert list(lay.res[:w.L]) == ref.res.tolist()
    assert list(lay.dense[:w.L]) == ref.dense.astype(int).tolist()
    assert list(lay.level_offset[:w.L]) == ref.offset.tolist()
    assert list(lay.level_size[:w.L]) == ref.size.tolist()
    assert lay.n_entries == ref.n_entries
    from oracle.step import ModelConfig
    cfg = ModelConfig(L=w.L, F=w.F, log2_T=w.log2_T, n_min=w.n_min, n_max=w.n_max, geo_out=w.geo_out,
                      colour=w.colour, shared_colour=w.shared_colour, n_slots=w.n_slots, view_dirs=w.view_dirs)
    assert lay.tile_params == cfg.tile_params()
    assert lay.n_params == cfg.n_params()
    assert lay.n_optimisers == cfg.n_optimisers()


@pytest.mark.parametrize("field,value", [("F", 3), ("L", 5), ("hidden", 32), ("geo_out", 8), ("n_slots", 5),
                                         ("log2_T", 30), ("precision", 7), ("n_min", 1), ("view_dirs", 1)])
def test_invalid_models_are_rejected(lib, field, value):
    m = snk.model_struct(8, 2, 14, 16, 256, 4, 0, 1, 1, snk.SNK_FP32)
    setattr(m, field, value)
    out = snk.SnkLayout()
    assert lib.snk_model_layout(ctypes.byref(m), ctypes.byref(out)) == snk.SNK_ERR_INVALID_ARG


def test_view_direction_models(lib):
    """The colour input [g | SH_16(d)] widens V1 by 16 columns; it needs a colour MLP
    and is not offered with the E4M3 first layer."""
    out = snk.SnkLayout()
    plain = snk.model_struct(8, 2, 14, 16, 256, 16, 1, 1, 2, snk.SNK_FP32)
    vd = snk.model_struct(8, 2, 14, 16, 256, 16, 1, 1, 2, snk.SNK_FP32, view_dirs=True)
    assert snk.layout(vd).colour_params == snk.layout(plain).colour_params + 64 * 16 == 64 * 32 + 64 * 64 + 3 * 64
    for prec, flag, ok in [(snk.SNK_MIXED, 1, True), (snk.SNK_MIXED_E4M3, 1, False), (snk.SNK_FP32, 2, False)]:
        m = snk.model_struct(8, 2, 14, 16, 256, 16, 1, 1, 2, prec)
        m.view_dirs = flag
        rc = lib.snk_model_layout(ctypes.byref(m), ctypes.byref(out))
        assert rc == (snk.SNK_OK if ok else snk.SNK_ERR_INVALID_ARG), (prec, flag)


def test_sample_capacity_bound(lib):
    """snk_max_samples: a ray's segments take clamp(rint(K_ray f_s), K_min, K_max) samples with
    the shares f_s summing to 1, so a brute-force maximum over share splits stays below the bound."""
    from synth import workloads as W
    rng = np.random.default_rng(0)
    for name in ["window2x2_full", "window2x2_fp8", "tiny_window", "tile512_full"]:
        w = W.get(name)
        win = snk.window_struct(w.window())
        sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max)
        bound = lib.snk_max_samples(ctypes.byref(win), ctypes.byref(sp), 1000)
        segs = 1 + (w.nx == 2) + (w.ny == 2)
        f = rng.dirichlet(np.full(segs, 0.3), 20000)
        f = np.concatenate([f, np.eye(segs), np.full((1, segs), 1.0 / segs)])
        k = np.clip(np.rint(w.K_ray * f.astype(np.float32)), w.K_min, w.K_max).sum(1)
        assert 1000 * k.max() <= bound - 4 * 128, (name, k.max(), bound)
        assert bound <= 1000 * segs * w.K_max + 4 * 128
    win = snk.window_struct(W.get("window2x2_full").window())
    uni = snk.sampler_struct(96, 64, 128, mode=snk.SNK_SAMPLE_UNIFORM)
    assert lib.snk_max_samples(ctypes.byref(win), ctypes.byref(uni), 10) == 10 * 96 + 4 * 128
    assert lib.snk_max_samples(None, ctypes.byref(uni), 10) == -1


def test_null_arguments_are_rejected_without_a_gpu(lib):
    assert lib.snk_model_layout(None, None) == snk.SNK_ERR_INVALID_ARG
    assert lib.snk_ctx_reserve(None, 1, 1) == snk.SNK_ERR_INVALID_ARG
    assert lib.snk_ctx_destroy(None) == snk.SNK_OK
    assert lib.snk_sync_status(None, None, None) == snk.SNK_ERR_INVALID_ARG
    assert lib.snk_wait_selftest(None, 0, None, None) == snk.SNK_ERR_INVALID_ARG


def test_a_missing_library_fails_loudly():
    """No fallback: without libsnk.so the binding raises (fresh interpreter, nothing loaded)."""
    import subprocess
    import sys
    code = ("from paper_2507_01631_b300 import snk\n"
            "try:\n    snk.load('/nonexistent/libsnk.so')\nexcept RuntimeError as e:\n"
            "    print('raised:', e)\n    raise SystemExit(0)\nraise SystemExit(1)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "not found" in r.stdout, (r.stdout, r.stderr)


def test_one_library_per_process(lib):
    assert snk.load() is lib
    with pytest.raises(RuntimeError):
        snk.load("/nonexistent/other/libsnk.so")


def test_static_sampler_refuses_bad_descriptors_before_any_cuda_call(lib):
    """The allocation-free sampler checks its window, sampler and cameras with the same rules
    as the context entry points (an RPC camera with a zero normalisation scale, a window whose
    slots are not a permutation, occupancy culling it has no scratch for), before touching the
    GPU: these run on a machine without one."""
    from synth import workloads as W
    w = W.get("tiny_window")
    cams = W.cameras(w)
    good = (snk.SnkCamera * len(cams))(*[snk.camera_struct(c) for c in cams])
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max)
    win = snk.window_struct(w.window())
    err = ctypes.create_string_buffer(256)

    def call(window, cam_arr, sampler):
        return lib.snk_sample_segments_static(ctypes.byref(window), cam_arr, len(cams), None, 0, ctypes.byref(sampler),
                                              *([None] * 9), 0, None, None, err, 256)
    bad_cams = (snk.SnkCamera * len(cams))(*[snk.camera_struct(c) for c in cams])
    bad_cams[1].kind = snk.SNK_CAM_RPC3
    bad_cams[1].scale[2] = 0.0
    assert call(win, bad_cams, sp) == snk.SNK_ERR_INVALID_ARG and b"zero normalisation scale" in err.value
    bad_win = snk.window_struct(w.window())
    bad_win.slot[1] = 0
    assert call(bad_win, good, sp) == snk.SNK_ERR_INVALID_ARG and b"permutation" in err.value
    occ = snk.sampler_struct(w.K_ray, w.K_min, w.K_max)
    occ.occ_res, occ.occupancy = 8, 1
    assert call(win, good, occ) == snk.SNK_ERR_INVALID_ARG and b"occupancy" in err.value
    pts = snk.sampler_struct(w.K_ray, 1, w.K_max, mode=snk.SNK_SAMPLE_POINTS)
    assert call(win, good, pts) == snk.SNK_ERR_INVALID_ARG and b"K_min >= 2" in err.value
