"""torch.autograd.Function wrappers over the stage entry points of libsnk.

Each wrapper pairs one forward entry point with its hand-written backward
(Sec. 4.1 encoding and MLPs, NeRF Eq. 3 compositing; the backward passes are
the analytic derivatives of those steps):

    SnkEncode     snk_encode / snk_encode_backward       table gradients
    SnkMLP        snk_mlp / snk_mlp_backward              weight and feature gradients
    SnkComposite  snk_composite / snk_composite_backward  sigma and colour gradients

The stage entry points compute in binary32 on the binary32 parameters,
whatever the model's precision field says; the fused mixed-precision step is
snk_train_step.  Every computation runs in the library's kernels: these
classes only allocate the output and gradient tensors and pass pointers.
Sample positions and times come from the sampler and carry no gradient
(the method differentiates neither the cameras nor the sample placement).

A Stages object binds a context, a model and a window; `sample()` runs the
ray / segment / sample stage and returns the batch the wrappers consume.
"""
import ctypes
from dataclasses import dataclass

import torch

from . import snk


@dataclass
class SampleBatch:
    """Output of snk_sample_segments for B rays, sample capacity `cap`
    (slot-major sample arrays; see the header for the layout)."""
    B: int
    cap: int
    ray_od: torch.Tensor
    ray_ok: torch.Tensor
    seg_slot: torch.Tensor
    seg_t: torch.Tensor
    seg_n: torch.Tensor
    seg_off: torch.Tensor
    smp_t: torch.Tensor
    smp_dt: torch.Tensor
    smp_xyz: torch.Tensor
    state: torch.Tensor


class Stages:
    """A context, a model and a window: what every stage call needs."""

    def __init__(self, ctx, model, window):
        self.ctx = ctx
        self.model = model
        self.window = window
        self.lay = snk.layout(model)
        self.in_dim = model.L * model.F

    def stream(self):
        return snk.stream_handle(torch.cuda.current_stream())

    def params_struct(self, params, grads=None):
        return snk.SnkParams(snk.ptr(params), None, snk.ptr(grads), None, None, None)

    def sample(self, pix, sampler, cap=None):
        """Rays, segments and samples of the packed pixels `pix` (int32 [B] on the device)."""
        B = int(pix.numel())
        n_seg = 1 + (self.window.nx == 2) + (self.window.ny == 2)
        if cap is None:
            cap = B * n_seg * sampler.K_max + 4 * 128
        dev = pix.device
        f32, i32, u8 = torch.float32, torch.int32, torch.uint8
        b = SampleBatch(
            B=B, cap=cap,
            ray_od=torch.zeros(6 * B, dtype=f32, device=dev),
            ray_ok=torch.zeros(B, dtype=u8, device=dev),
            seg_slot=torch.zeros(3 * B, dtype=u8, device=dev),
            seg_t=torch.zeros(6 * B, dtype=f32, device=dev),
            seg_n=torch.zeros(3 * B, dtype=i32, device=dev),
            seg_off=torch.zeros(3 * B, dtype=i32, device=dev),
            smp_t=torch.zeros(max(cap, 1), dtype=f32, device=dev),
            smp_dt=torch.zeros(max(cap, 1), dtype=f32, device=dev),
            smp_xyz=torch.zeros(3 * max(cap, 1), dtype=f32, device=dev),
            state=torch.zeros(snk.STATE_WORDS, dtype=i32, device=dev))
        self.ctx.call("snk_sample_segments", ctypes.byref(self.window), snk.ptr(pix), B, ctypes.byref(sampler),
                      snk.ptr(b.ray_od), snk.ptr(b.ray_ok), snk.ptr(b.seg_slot), snk.ptr(b.seg_t),
                      snk.ptr(b.seg_n), snk.ptr(b.seg_off), snk.ptr(b.smp_t), snk.ptr(b.smp_dt),
                      snk.ptr(b.smp_xyz), cap, snk.ptr(b.state), self.stream())
        return b

    # convenience: the whole differentiable forward of a sampled batch
    def render(self, params, batch):
        feat = SnkEncode.apply(params, batch.smp_xyz, batch.state, self)
        sigma_rgb = SnkMLP.apply(params, feat, batch.state, self)
        return SnkComposite.apply(sigma_rgb, batch.smp_t, batch.smp_dt, batch.seg_n, batch.seg_off, self)


def _check(params, stages):
    if params.dtype != torch.float32 or not params.is_cuda or not params.is_contiguous():
        raise TypeError("params must be a contiguous float32 CUDA tensor")
    if params.numel() != stages.lay.n_params:
        raise ValueError("params has %d elements, the model's layout %d" % (params.numel(), stages.lay.n_params))


class SnkEncode(torch.autograd.Function):
    """feat [cap, L*F] = hash encoding of the slot-major samples (tables of `params`)."""

    @staticmethod
    def forward(ctx, params, smp_xyz, state, stages):
        _check(params, stages)
        cap = smp_xyz.numel() // 3
        feat = torch.zeros(cap, stages.in_dim, dtype=torch.float32, device=params.device)
        ps = stages.params_struct(params)
        stages.ctx.call("snk_encode", ctypes.byref(stages.model), ctypes.byref(ps), snk.ptr(smp_xyz),
                        snk.ptr(state), cap, snk.ptr(feat), None, stages.stream())
        ctx.save_for_backward(params, smp_xyz, state)
        ctx.stages = stages
        return feat

    @staticmethod
    def backward(ctx, dfeat):
        params, smp_xyz, state = ctx.saved_tensors
        stages = ctx.stages
        grads = torch.zeros_like(params)
        ps = stages.params_struct(params, grads)
        cap = smp_xyz.numel() // 3
        stages.ctx.call("snk_encode_backward", ctypes.byref(stages.model), ctypes.byref(ps), snk.ptr(smp_xyz),
                        snk.ptr(state), cap, snk.ptr(dfeat.contiguous()), stages.stream())
        return grads, None, None, None


class SnkMLP(torch.autograd.Function):
    """sigma_rgb [cap, 4] = (sigma, r, g, b) of the density and colour MLPs on feat."""

    @staticmethod
    def forward(ctx, params, feat, state, stages):
        _check(params, stages)
        feat = feat.contiguous()
        cap = feat.shape[0]
        out = torch.zeros(cap, 4, dtype=torch.float32, device=params.device)
        ps = stages.params_struct(params)
        stages.ctx.call("snk_mlp", ctypes.byref(stages.model), ctypes.byref(ps), snk.ptr(feat), snk.ptr(state),
                        cap, snk.ptr(out), stages.stream())
        ctx.save_for_backward(params, feat, state)
        ctx.stages = stages
        return out

    @staticmethod
    def backward(ctx, dout):
        params, feat, state = ctx.saved_tensors
        stages = ctx.stages
        grads = torch.zeros_like(params)
        dfeat = torch.zeros_like(feat)
        ps = stages.params_struct(params, grads)
        stages.ctx.call("snk_mlp_backward", ctypes.byref(stages.model), ctypes.byref(ps), snk.ptr(feat),
                        snk.ptr(state), feat.shape[0], snk.ptr(dout.contiguous()), snk.ptr(dfeat), stages.stream())
        return grads, dfeat, None, None


class SnkComposite(torch.autograd.Function):
    """Front-to-back compositing of B rays: returns rgb [B, 3], depth [B] and
    opacity [B].  Only rgb is differentiable (the method's loss is on colour)."""

    @staticmethod
    def forward(ctx, sigma_rgb, smp_t, smp_dt, seg_n, seg_off, stages):
        sigma_rgb = sigma_rgb.contiguous()
        B = seg_n.numel() // 3
        out = torch.zeros(B, 5, dtype=torch.float32, device=sigma_rgb.device)
        stages.ctx.call("snk_composite", snk.ptr(sigma_rgb), snk.ptr(smp_t), snk.ptr(smp_dt), snk.ptr(seg_n),
                        snk.ptr(seg_off), B, snk.ptr(out), None, stages.stream())
        ctx.save_for_backward(sigma_rgb, smp_t, smp_dt, seg_n, seg_off)
        ctx.stages = stages
        rgb, depth, opacity = out[:, :3].contiguous(), out[:, 3].contiguous(), out[:, 4].contiguous()
        ctx.mark_non_differentiable(depth, opacity)
        return rgb, depth, opacity

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_opacity):
        sigma_rgb, smp_t, smp_dt, seg_n, seg_off = ctx.saved_tensors
        stages = ctx.stages
        B = seg_n.numel() // 3
        d = torch.zeros_like(sigma_rgb)
        if g_rgb is not None:
            stages.ctx.call("snk_composite_backward", snk.ptr(sigma_rgb), snk.ptr(smp_t), snk.ptr(smp_dt),
                            snk.ptr(seg_n), snk.ptr(seg_off), B, snk.ptr(g_rgb.contiguous()), snk.ptr(d),
                            stages.stream())
        return d, None, None, None, None, None
