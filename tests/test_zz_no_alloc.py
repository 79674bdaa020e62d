"""The allocation-free sampling entry point, for callers that cannot allocate
device memory (their own allocator owns it, or cudaMalloc is not allowed where
they run): called through the C ABI, it must give exactly the results of the
ordinary snk_sample_segments on the same inputs, on two calls in a row with
different batches (so a stale scratch from the first call would show), and it
must refuse batches larger than its fixed scratch.  Collected last so that a
failure here does not stop the rest of the GPU tests."""
import ctypes
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from gpu_util import make_case
from synth import workloads as W

pytestmark = pytest.mark.gpu
FIELDS = ("ray_od", "ray_ok", "seg_slot", "seg_t", "seg_n", "seg_off", "smp_t", "smp_dt", "smp_xyz")


@pytest.fixture(scope="module")
def lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    return snk.load()


def _buffers(B, cap):
    f32, i32, u8 = torch.float32, torch.int32, torch.uint8
    return {"ray_od": torch.zeros(6 * B, dtype=f32, device="cuda"), "ray_ok": torch.zeros(B, dtype=u8, device="cuda"),
            "seg_slot": torch.zeros(3 * B, dtype=u8, device="cuda"), "seg_t": torch.zeros(6 * B, dtype=f32, device="cuda"),
            "seg_n": torch.zeros(3 * B, dtype=i32, device="cuda"), "seg_off": torch.zeros(3 * B, dtype=i32, device="cuda"),
            "smp_t": torch.zeros(cap, dtype=f32, device="cuda"), "smp_dt": torch.zeros(cap, dtype=f32, device="cuda"),
            "smp_xyz": torch.zeros(3 * cap, dtype=f32, device="cuda"),
            "state": torch.zeros(snk.STATE_WORDS, dtype=i32, device="cuda")}


def _args(g):
    return [snk.ptr(g[k]) for k in FIELDS]


def _run_both(lib, ctx, case, seed, iteration):
    w = case.w
    B = len(case.pix)
    cap = B * (1 + (w.nx == 2) + (w.ny == 2)) * w.K_max + 512
    ws = snk.window_struct(w.window())
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, seed, iteration)
    pix = torch.from_numpy(case.pix.view(np.int32).copy()).cuda()
    ref = _buffers(B, cap)
    ctx.set_views(case.cams)
    ctx.call("snk_sample_segments", ctypes.byref(ws), snk.ptr(pix), B, ctypes.byref(sp), *_args(ref), cap,
             snk.ptr(ref["state"]), None)
    new = _buffers(B, cap)
    cams = (snk.SnkCamera * len(case.cams))(*[snk.camera_struct(c) for c in case.cams])
    err = ctypes.create_string_buffer(256)
    rc = lib.snk_sample_segments_static(ctypes.byref(ws), cams, len(case.cams), snk.ptr(pix), B, ctypes.byref(sp),
                                        *_args(new), cap, snk.ptr(new["state"]), None, err, 256)
    assert rc == snk.SNK_OK, err.value
    torch.cuda.synchronize()
    return ref, new


@pytest.mark.parametrize("name,n_rays", [("tiny_window", 160), ("tile512_full", 3000)])
def test_static_entry_point_matches_the_allocating_one_twice(lib, name, n_rays):
    ctx = snk.Context(0)
    try:
        for call, seed in enumerate((11, 12)):
            case = make_case(name, n_rays=n_rays, seed=seed, with_targets=False)
            ref, new = _run_both(lib, ctx, case, seed=7 + call, iteration=call)
            for k in FIELDS + ("state",):
                a, b = ref[k].cpu().numpy(), new[k].cpu().numpy()
                assert np.array_equal(a, b), "call %d: %s differs" % (call + 1, k)
            assert int(new["state"][3].item()) > 0
    finally:
        ctx.close()


def test_static_entry_point_rejects_batches_beyond_its_scratch(lib):
    case = make_case("tiny_tile", n_rays=8, with_targets=False)
    w = case.w
    ws = snk.window_struct(w.window())
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 0, 0)
    cams = (snk.SnkCamera * len(case.cams))(*[snk.camera_struct(c) for c in case.cams])
    err = ctypes.create_string_buffer(256)
    g = _buffers(8, 1024)
    rc = lib.snk_sample_segments_static(ctypes.byref(ws), cams, len(case.cams), snk.ptr(g["ray_ok"]), 65537,
                                        ctypes.byref(sp), *_args(g), 1024, snk.ptr(g["state"]), None, err, 256)
    assert rc == snk.SNK_ERR_INVALID_ARG
    assert b"65536" in err.value


def _static_call(lib, w, cams, pix, sp, g, cap, stream):
    cam_arr = (snk.SnkCamera * len(cams))(*[snk.camera_struct(c) for c in cams])
    err = ctypes.create_string_buffer(256)
    rc = lib.snk_sample_segments_static(ctypes.byref(snk.window_struct(w.window())), cam_arr, len(cams),
                                        snk.ptr(pix), len(pix), ctypes.byref(sp), *_args(g), cap,
                                        snk.ptr(g["state"]), snk.stream_handle(stream), err, 256)
    return rc, err.value


def test_static_calls_queued_on_one_stream_match_the_allocating_one(lib):
    """Three calls with different windows, cameras, batches and seeds queued on one stream
    before a single synchronise (each with its own output buffers): the host staging of the
    cameras is reused by the next call while the earlier copies may still be in flight, and
    every call must still sample with its own cameras."""
    base = W.get("tile512_full")
    jobs = []
    for w, seed in [(dataclasses.replace(base, n_rays=2000), 7), (dataclasses.replace(base, n_rays=2500, seed=5), 8),
                    (dataclasses.replace(W.get("tiny_window"), n_rays=160), 9)]:
        cams = W.cameras(w)
        pix_h = W.batch(w, cams, 40 + seed)
        jobs.append((w, cams, pix_h, snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, seed, seed)))
    stream = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(stream):
        for w, cams, pix_h, sp in jobs:
            B = len(pix_h)
            cap = B * (1 + (w.nx == 2) + (w.ny == 2)) * w.K_max + 512
            pix = torch.from_numpy(pix_h.view(np.int32).copy()).cuda()
            g = _buffers(B, cap)
            rc, msg = _static_call(lib, w, cams, pix, sp, g, cap, stream)
            assert rc == snk.SNK_OK, msg
            outs.append((g, pix, cap))
    stream.synchronize()
    ctx = snk.Context(0)
    try:
        for (w, cams, pix_h, sp), (g, pix, cap) in zip(jobs, outs):
            ref = _buffers(len(pix_h), cap)
            ctx.set_views(cams)
            ctx.call("snk_sample_segments", ctypes.byref(snk.window_struct(w.window())), snk.ptr(pix), len(pix_h),
                     ctypes.byref(sp), *_args(ref), cap, snk.ptr(ref["state"]), None)
            torch.cuda.synchronize()
            for k in FIELDS + ("state",):
                assert np.array_equal(ref[k].cpu().numpy(), g[k].cpu().numpy()), (w.name, k)
            assert int(g["state"][3].item()) > 0
    finally:
        ctx.close()


def test_static_entry_point_refuses_a_capturing_stream(lib):
    """A call on a stream that is capturing a CUDA graph is refused before anything is queued
    (its camera copy would replay a stale host array)."""
    case = make_case("tiny_tile", n_rays=8, with_targets=False)
    w = case.w
    sp = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 0, 0)
    pix = torch.from_numpy(case.pix.view(np.int32).copy()).cuda()
    g = _buffers(8, 1024)
    x = torch.zeros(16, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rc, msg = _static_call(lib, w, case.cams, pix, sp, g, 1024, torch.cuda.current_stream())
        x.add_(1.0)
    assert rc == snk.SNK_ERR_INVALID_ARG and b"captur" in msg, (rc, msg)
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    # outside the capture the same call runs
    rc, msg = _static_call(lib, w, case.cams, pix, sp, g, 1024, None)
    assert rc == snk.SNK_OK, msg
    torch.cuda.synchronize()
