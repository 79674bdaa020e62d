"""ctypes binding of libsnk (include/snk.h): struct mirrors and the C entry points
under their C names.  Argument marshalling only -- every step of the method
runs in the library's CUDA kernels.  Device buffers are passed as torch
tensors (their data_ptr()) or raw integers; streams as torch streams or
raw handles.  The binding fails loudly if libsnk.so is missing: there is no
fallback implementation.
"""
import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_uint32,
                    c_void_p)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsnk.so")

SNK_OK, SNK_ERR_INVALID_ARG, SNK_ERR_CUDA, SNK_ERR_OOM, SNK_ERR_TIMEOUT, SNK_ERR_DEVICE_CHECK, SNK_ERR_OVERFLOW = range(7)
SNK_CAM_AFFINE, SNK_CAM_RPC3 = 0, 1
SNK_FP32, SNK_MIXED, SNK_MIXED_E4M3 = 0, 1, 2
SNK_SAMPLE_SEGMENTS, SNK_SAMPLE_UNIFORM, SNK_SAMPLE_POINTS = 0, 1, 2
STATUS_OVERFLOW, STATUS_CHECK, STATUS_TIMEOUT = 1, 2, 4


class SnkCamera(Structure):
    _fields_ = [("kind", c_int32), ("width", c_int32), ("height", c_int32), ("crop_r0", c_int32),
                ("crop_c0", c_int32), ("crop_h", c_int32), ("crop_w", c_int32), ("reserved", c_int32),
                ("a", c_double * 4), ("b", c_double * 4), ("off", c_double * 5), ("scale", c_double * 5),
                ("coef", (c_double * 20) * 4)]


class SnkWindow(Structure):
    _fields_ = [("origin", c_double * 3), ("tile_size", c_double * 3), ("scene_lo", c_double * 3),
                ("scene_hi", c_double * 3), ("nx", c_int32), ("ny", c_int32), ("slot", c_int32 * 4)]


class SnkModel(Structure):
    _fields_ = [(n, c_int32) for n in ("L", "F", "log2_T", "n_min", "n_max", "hidden", "geo_out", "colour",
                                        "shared_colour", "n_slots", "precision", "view_dirs")]


class SnkLayout(Structure):
    _fields_ = [("res", c_int32 * 32), ("dense", c_int32 * 32), ("level_offset", c_int64 * 32),
                ("level_size", c_int64 * 32), ("n_entries", c_int64), ("grid_params", c_int64),
                ("tile_params", c_int64), ("colour_params", c_int64), ("n_params", c_int64),
                ("n_optimisers", c_int32), ("n_colour_blocks", c_int32)]


class SnkSampler(Structure):
    _fields_ = [("K_ray", c_int32), ("K_min", c_int32), ("K_max", c_int32), ("render", c_int32),
                ("seed", c_uint32), ("iteration", c_uint32), ("occ_res", c_int32), ("mode", c_int32),
                ("occupancy", c_void_p)]


class SnkAdam(Structure):
    _fields_ = [("lr", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float), ("l2_mlp", c_float)]


class SnkParams(Structure):
    _fields_ = [("params", c_void_p), ("params_lp", c_void_p), ("grads", c_void_p), ("adam_m", c_void_p),
                ("adam_v", c_void_p), ("adam_step", c_void_p)]


class SnkState(Structure):
    _fields_ = [("loss", c_float), ("loss_scale", c_float), ("n_accepted", c_uint32), ("n_samples", c_uint32),
                ("status", c_uint32), ("good_steps", c_int32), ("iteration", c_uint32),
                ("slot_base", c_uint32 * 5), ("slot_count", c_uint32 * 4), ("nonfinite", c_uint32),
                ("bwd_mode", c_uint32), ("reserved", c_uint32)]


class SnkTuning(Structure):
    _fields_ = [("tc_fwd_ctas", c_int32), ("tc_fwd_levels", c_int32), ("fp32_ctas", c_int32),
                ("composite_threads", c_int32), ("sampler_threads", c_int32), ("tuned", c_int32),
                ("tc_bwd_saved", c_int32), ("tc_fwd_split", c_int32)]


STRUCTS = [SnkCamera, SnkWindow, SnkModel, SnkLayout, SnkSampler, SnkAdam, SnkParams, SnkState, SnkTuning]
STATE_WORDS = ctypes.sizeof(SnkState) // 4

_P = c_void_p
# name -> (restype, argtypes)
SIGNATURES = {
    "snk_version": (c_char_p, []),
    "snk_abi_sizes": (c_int, [POINTER(c_int64), c_int]),
    "snk_model_layout": (c_int, [POINTER(SnkModel), POINTER(SnkLayout)]),
    "snk_ctx_create": (c_int, [c_int, POINTER(c_void_p)]),
    "snk_ctx_destroy": (c_int, [_P]),
    "snk_ctx_reserve": (c_int, [_P, c_int64, c_int64]),
    "snk_ctx_set_act_budget": (c_int, [_P, c_int64]),
    "snk_params_refresh_lp": (c_int, [_P, POINTER(SnkModel), POINTER(SnkParams), _P]),
    "snk_max_samples": (c_int64, [POINTER(SnkWindow), POINTER(SnkSampler), c_int64]),
    "snk_last_error": (c_char_p, [_P]),
    "snk_set_views": (c_int, [_P, POINTER(SnkCamera), c_int, POINTER(c_void_p), _P]),
    "snk_sample_segments": (c_int, [_P, POINTER(SnkWindow), _P, c_int, POINTER(SnkSampler), _P, _P, _P, _P, _P,
                                    _P, _P, _P, _P, c_int64, _P, _P]),
    "snk_encode": (c_int, [_P, POINTER(SnkModel), POINTER(SnkParams), _P, _P, c_int64, _P, _P, _P]),
    "snk_encode_backward": (c_int, [_P, POINTER(SnkModel), POINTER(SnkParams), _P, _P, c_int64, _P, _P]),
    "snk_mlp": (c_int, [_P, POINTER(SnkModel), POINTER(SnkParams), _P, _P, c_int64, _P, _P]),
    "snk_mlp_backward": (c_int, [_P, POINTER(SnkModel), POINTER(SnkParams), _P, _P, c_int64, _P, _P, _P]),
    "snk_composite": (c_int, [_P, _P, _P, _P, _P, _P, c_int, _P, _P, _P]),
    "snk_composite_backward": (c_int, [_P, _P, _P, _P, _P, _P, c_int, _P, _P, _P]),
    "snk_train_step": (c_int, [_P, POINTER(SnkModel), POINTER(SnkWindow), _P, c_int, POINTER(SnkSampler),
                               POINTER(SnkAdam), POINTER(SnkParams), _P, _P, _P]),
    "snk_render": (c_int, [_P, POINTER(SnkModel), POINTER(SnkWindow), _P, c_int, POINTER(SnkSampler),
                           POINTER(SnkParams), _P, _P, _P]),
    "snk_sync_status": (c_int, [_P, _P, _P]),
    "snk_quantize_e4m3": (c_int, [_P, _P, c_int64, c_float, _P, _P]),
    "snk_build_crops": (c_int, [_P, POINTER(SnkWindow), c_int, _P, _P, _P]),
    "snk_ray_pool": (c_int, [_P, POINTER(SnkWindow), _P, _P, c_int64, _P, _P]),
    "snk_draw_batch": (c_int, [_P, _P, _P, c_int, c_uint32, c_uint32, _P, _P]),
    "snk_occupancy_update": (c_int, [_P, POINTER(SnkModel), POINTER(SnkParams), _P, _P, c_int, c_float, c_float,
                                     c_uint32, c_uint32, _P]),
    "snk_tile_bytes": (c_int, [POINTER(SnkModel), POINTER(c_int64)]),
    "snk_tile_park": (c_int, [_P, POINTER(SnkModel), POINTER(SnkParams), c_int, _P, _P]),
    "snk_tile_unpark": (c_int, [_P, POINTER(SnkModel), POINTER(SnkParams), c_int, _P, _P]),
    "snk_get_tuning": (c_int, [_P, POINTER(SnkTuning)]),
    "snk_set_tuning": (c_int, [_P, POINTER(SnkTuning)]),
    "snk_autotune": (c_int, [_P, POINTER(SnkModel), POINTER(SnkWindow), _P, c_int, POINTER(SnkSampler),
                             POINTER(SnkParams), _P, POINTER(SnkTuning)]),
    "snk_sample_segments_static": (c_int, [POINTER(SnkWindow), POINTER(SnkCamera), c_int, _P, c_int,
                                           POINTER(SnkSampler), _P, _P, _P, _P, _P, _P, _P, _P, _P, c_int64, _P, _P,
                                           c_char_p, c_int]),
    "snk_launch_count": (c_int64, []),
    "snk_l2_reduction_probe": (c_int, [_P, _P, c_int64, c_int64, c_int, c_uint32, _P]),
    "snk_wait_selftest": (c_int, [_P, c_int, _P, _P]),
    "snk_stage_timing": (c_int, [_P, c_int]),
    "snk_stage_times": (c_int, [_P, POINTER(c_double), POINTER(c_int64), c_int]),
}
STAGES = ("rays_segments_samples", "field_forward", "render_loss_backward", "field_backward", "adam")

_lib = None
_lib_path = None


def load(path=None):
    """Load libsnk.so (built by paper_2507_01631_b300.build; path None = the in-tree one) and
    declare signatures.  One library per process: once one is loaded, load() returns it, and
    asking explicitly for another path is an error."""
    global _lib, _lib_path
    if _lib is not None:
        if path is not None and os.path.abspath(path) != _lib_path:
            raise RuntimeError("libsnk already loaded from %s, not %s" % (_lib_path, os.path.abspath(path)))
        return _lib
    path = os.path.abspath(LIB_PATH if path is None else path)
    if not os.path.exists(path):
        raise RuntimeError("libsnk.so not found at %s: run `python -m paper_2507_01631_b300.build`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib, _lib_path = lib, path
    return lib


def ptr(x):
    """Device/host address of a torch tensor, an int, or None (NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class SnkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libsnk error %d: %s" % (code, msg))
        self.code = code


def check(rc, ctx=None):
    if rc != SNK_OK:
        msg = load().snk_last_error(ctx).decode() if ctx else ""
        raise SnkError(rc, msg)
    return rc


# ---- struct builders from plain Python / synth objects ------------------------
def camera_struct(cam):
    c = SnkCamera()
    c.kind = int(cam.kind)
    c.width, c.height = int(cam.width), int(cam.height)
    c.crop_r0, c.crop_c0, c.crop_h, c.crop_w = (int(v) for v in cam.crop)
    for i in range(4):
        c.a[i] = float(cam.a[i])
        c.b[i] = float(cam.b[i])
    for i in range(5):
        c.off[i] = float(cam.off[i])
        c.scale[i] = float(cam.scale[i])
    for r in range(4):
        for k in range(20):
            c.coef[r][k] = float(cam.coef[r][k])
    return c


def window_struct(win):
    w = SnkWindow()
    for a in range(3):
        w.origin[a] = float(win.origin[a])
        w.tile_size[a] = float(win.tile_size[a])
        w.scene_lo[a] = float(win.scene_lo[a])
        w.scene_hi[a] = float(win.scene_hi[a])
    w.nx, w.ny = int(win.nx), int(win.ny)
    for q in range(4):
        w.slot[q] = int(win.slot[q]) if q < len(win.slot) else 0
    return w


def model_struct(L, F, log2_T, n_min, n_max, geo_out, colour, shared_colour, n_slots, precision, hidden=64,
                 view_dirs=False):
    return SnkModel(L, F, log2_T, n_min, n_max, hidden, geo_out, int(colour), int(shared_colour), n_slots, precision,
                    int(view_dirs))


def sampler_struct(K_ray, K_min, K_max, render=0, seed=0, iteration=0, occupancy=None, occ_res=0, mode=0):
    """occupancy: device uint8 tensor [n_slots][occ_res^3] of occupied flags (culling), or None.
    The struct keeps the tensor's address only: the caller keeps the tensor alive while it is used.
    mode: SNK_SAMPLE_SEGMENTS, SNK_SAMPLE_UNIFORM or SNK_SAMPLE_POINTS."""
    return SnkSampler(K_ray, K_min, K_max, render, seed & 0xFFFFFFFF, iteration & 0xFFFFFFFF,
                      occ_res if occupancy is not None else 0, mode, ptr(occupancy))


def adam_struct(lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15, l2_mlp=1e-6):
    return SnkAdam(lr, beta1, beta2, eps, l2_mlp)


def layout(model):
    out = SnkLayout()
    check(load().snk_model_layout(ctypes.byref(model), ctypes.byref(out)))
    return out


class Context:
    """Owns one snk_ctx on a device.  Creating it makes that device current; later calls run
    on the calling thread's current device, which must be the context's (torch.cuda.set_device
    or torch.cuda.device(ctx.device) when several devices are in use)."""

    def __init__(self, device=0):
        self.lib = load()
        h = c_void_p()
        check(self.lib.snk_ctx_create(device, ctypes.byref(h)))
        self.h = h.value
        self.device = int(device)
        self._keep = []

    def close(self):
        if self.h:
            self.lib.snk_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def call(self, name, *args):
        return check(getattr(self.lib, name)(self.h, *args), self.h)

    def reserve(self, max_rays, max_samples):
        self.call("snk_ctx_reserve", max_rays, max_samples)

    def set_act_budget(self, nbytes):
        """Most bytes of stored activations the context may hold (snk_ctx_set_act_budget); a
        step that needs more recomputes them in its backward.  None or < 0: no budget."""
        self.call("snk_ctx_set_act_budget", -1 if nbytes is None else int(nbytes))

    def max_samples(self, window, sampler, n_rays):
        """The sample capacity a step of n_rays rays sizes its workspace for (snk_max_samples)."""
        return int(self.lib.snk_max_samples(ctypes.byref(window), ctypes.byref(sampler), int(n_rays)))

    def set_views(self, cams, crops=None, stream=None):
        arr = (SnkCamera * len(cams))(*[camera_struct(c) for c in cams])
        cp = None
        if crops is not None:
            cp = (c_void_p * len(cams))(*[ptr(x) for x in crops])
        self.call("snk_set_views", arr, len(cams), cp, stream_handle(stream))
        self._keep = [arr, crops]

    def stage_timing(self, enable=True):
        self.call("snk_stage_timing", 1 if enable else 0)

    def stage_times(self):
        ms = (c_double * 5)()
        calls = (c_int64 * 5)()
        self.call("snk_stage_times", ms, calls, 5)
        return {n: (ms[i], calls[i]) for i, n in enumerate(STAGES)}

    def tuning(self):
        t = SnkTuning()
        self.call("snk_get_tuning", ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in SnkTuning._fields_ if k != "reserved"}

    def set_tuning(self, **values):
        t = SnkTuning()
        self.call("snk_get_tuning", ctypes.byref(t))
        names = {k for k, _ in SnkTuning._fields_}
        for k, v in values.items():
            if k not in names:
                raise KeyError("unknown launch-shape field %r" % k)
            setattr(t, k, int(v))
        self.call("snk_set_tuning", ctypes.byref(t))

    def autotune(self, model, window, pix, sampler, params_struct, stream=None):
        """Pick the context's launch shapes on this batch (snk_autotune); returns them."""
        t = SnkTuning()
        self.call("snk_autotune", ctypes.byref(model), ctypes.byref(window), ptr(pix), int(pix.numel()),
                  ctypes.byref(sampler), ctypes.byref(params_struct), stream_handle(stream), ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in SnkTuning._fields_ if k != "reserved"}

    def sync_status(self, state, stream=None):
        return self.lib.snk_sync_status(self.h, ptr(state), stream_handle(stream))
