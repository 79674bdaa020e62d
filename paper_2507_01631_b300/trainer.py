"""Tensor plumbing around libsnk: allocates the trainable state and the per-step
device state as torch tensors and calls snk_train_step / snk_render.  No step
of the method is computed here."""
import ctypes

import numpy as np
import torch

from . import snk

STATE_FIELDS = {"loss": (0, "f"), "loss_scale": (1, "f"), "n_accepted": (2, "u"), "n_samples": (3, "u"),
                "status": (4, "u"), "good_steps": (5, "i"), "iteration": (6, "u"), "bwd_mode": (17, "u")}
BWD_MODES = {0: "binary32", 1: "stored activations", 2: "recomputed activations"}


def model_from_workload(w, precision=None, hidden=64):
    if precision is None:
        precision = snk.SNK_FP32
        if w.mixed:
            precision = snk.SNK_MIXED_E4M3 if getattr(w, "first_layer", "f16") == "e4m3" else snk.SNK_MIXED
    prec = precision
    return snk.model_struct(w.L, w.F, w.log2_T, w.n_min, w.n_max, w.geo_out, w.colour, w.shared_colour,
                            w.n_slots, prec, hidden, view_dirs=getattr(w, "view_dirs", False))


class Trainer:
    """One model (1 tile or a 2x2 window) with its Adam state on a CUDA device."""

    def __init__(self, ctx, model, window, sampler, init_params, adam=None, loss_scale=None, device="cuda"):
        self.ctx = ctx
        self.model = model
        self.window = window
        self.sampler = sampler
        self.adam = adam or snk.adam_struct()
        self.lay = snk.layout(model)
        n = self.lay.n_params
        p = torch.as_tensor(np.asarray(init_params, np.float32)).to(device)
        assert p.numel() == n, (p.numel(), n)
        self.params = p.contiguous()
        self.mixed = model.precision != snk.SNK_FP32
        # FP16 working copy (mixed precision): written by the library from the master weights
        self.params_lp = torch.empty(n, dtype=torch.int16, device=device) if self.mixed else None
        self.grads = torch.zeros(n, dtype=torch.float32, device=device)
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.steps = torch.zeros(self.lay.n_optimisers, dtype=torch.int32, device=device)
        self.state = torch.zeros(snk.STATE_WORDS, dtype=torch.int32, device=device)
        scale = loss_scale if loss_scale is not None else (65536.0 if self.mixed else 1.0)
        self.state.view(torch.float32)[1] = scale
        self.p_struct = snk.SnkParams(snk.ptr(self.params), snk.ptr(self.params_lp), snk.ptr(self.grads),
                                      snk.ptr(self.m), snk.ptr(self.v), snk.ptr(self.steps))
        if self.mixed:
            self.refresh_lp()

    def refresh_lp(self, stream=None):
        """Rewrite the FP16 working copy from the binary32 master weights (snk_params_refresh_lp),
        e.g. after the caller changed self.params."""
        self.ctx.call("snk_params_refresh_lp", ctypes.byref(self.model), ctypes.byref(self.p_struct),
                      snk.stream_handle(stream))

    def train_step(self, pix, out=None, stream=None):
        self.ctx.call("snk_train_step", ctypes.byref(self.model), ctypes.byref(self.window), snk.ptr(pix),
                      int(pix.numel()), ctypes.byref(self.sampler), ctypes.byref(self.adam),
                      ctypes.byref(self.p_struct), snk.ptr(self.state), snk.ptr(out), snk.stream_handle(stream))

    def render(self, pix, out, stream=None):
        self.ctx.call("snk_render", ctypes.byref(self.model), ctypes.byref(self.window), snk.ptr(pix),
                      int(pix.numel()), ctypes.byref(self.sampler), ctypes.byref(self.p_struct),
                      snk.ptr(self.state), snk.ptr(out), snk.stream_handle(stream))

    def autotune(self, pix, stream=None):
        """Pick the context's launch shapes on this batch (snk_autotune); the
        trainer's parameters, gradients and Adam state are not modified."""
        return self.ctx.autotune(self.model, self.window, pix, self.sampler, self.p_struct, stream)

    def read_state(self):
        s = self.state.cpu().numpy()
        out = {}
        for k, (i, t) in STATE_FIELDS.items():
            out[k] = float(s[i:i + 1].view(np.float32)[0]) if t == "f" else int(s[i:i + 1].view(np.uint32)[0])
        out["bwd_mode_name"] = BWD_MODES.get(out["bwd_mode"], "?")
        out["slot_base"] = s[7:12].view(np.uint32).tolist()
        out["slot_count"] = s[12:16].view(np.uint32).tolist()
        return out
