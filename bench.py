"""Benchmark of the Snake-NeRF training step on B300: train samples/s for the
full step (rays, segments, samples, encoding, MLPs, rendering, loss,
backward, Adam) on synthetic satellite-like data.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision fp32|mixed|both] [--impl ours|reference]

One JSON line on stdout (rank 0).  With N > 1 (torchrun) every rank trains an
independent replica on its own GPU ("replicas only": the step has no
exchange); value = samples of all ranks / max elapsed over ranks.
`--impl reference` times the FP64 CPU oracle on bounded samples of the same
workload (the reference arm; rank 0 only).
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import workloads as W  # noqa: E402
import synth  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}
METRIC = "train samples/s (fwd+bwd+Adam), FP32 per-tile vs mixed 2x2-batched, equal PSNR"
N_BATCHES = 4  # distinct ray batches cycled through the timed steps


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="window2x2_full")
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed"])
    ap.add_argument("--graph", type=int, default=1, help="also time replays of the step captured as a CUDA graph")
    ap.add_argument("--compare-fp32", type=int, default=1,
                    help="also time the binary32 per-tile path on the same workload (mixed runs only)")
    ap.add_argument("--fp32-steps", type=int, default=3)
    ap.add_argument("--rays", type=int, default=0, help="override the workload's rays per step (profiling)")
    ap.add_argument("--bwd-saved", default="auto", choices=["auto", "0", "1"],
                    help="tensor-core backward: 1 reads the activations the forward stored, 0 recomputes "
                         "the forward, auto lets the autotuner (or the default) decide")
    ap.add_argument("--fwd-split", default="auto", choices=["auto", "0", "1"],
                    help="tensor-core forward: 1 dedicated gather warps, 0 every thread gathers then runs "
                         "the chain, auto lets the autotuner (or the default) decide")
    ap.add_argument("--sampler-mode", default="segments", choices=["segments", "uniform", "points"],
                    help="variant: the per-tile segmented sampler, the NeRF-XL uniform distribution, "
                         "or point samples with backward-difference deltas")
    ap.add_argument("--view-dirs", type=int, default=0,
                    help="variant: colour input [g | SH_16(ray direction)] instead of g")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-rays", type=int, default=256, help="rays per oracle sample (CPU baseline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stage-timing", type=int, default=1)
    ap.add_argument("--autotune", type=int, default=1, help="pick the launch shapes on the first batch first")
    ap.add_argument("--red-ceiling", type=int, default=1,
                    help="also time the stand-alone reduction probe (the peak of the reduction roofline)")
    return ap.parse_args()


def peaks():
    if os.path.exists(PEAKS_FILE):
        d = json.load(open(PEAKS_FILE))
        d["source"] = "measured"
        return d
    d = dict(FALLBACK_PEAKS)
    d["source"] = "fallback"
    return d


# ---- per-sample algorithmic work ----------------------------------------------------
def mlp_flops_per_sample(w):
    IN, H, G = w.L * w.F, 64, w.geo_out
    CIN = G + (16 if w.view_dirs else 0)  # colour input: g, or [g | SH_16(direction)]
    mac = IN * H + H * H + H * G + ((CIN * H + H * H + H * 3) if w.colour else 0)
    return 2 * mac


def act_bytes_per_sample(w):
    """FP16 high parts of the activations a training forward stores for its
    backward: h1, h2 (64 each) and, with a colour net, g (16, 32 with view
    directions), c1, c2 (64 each)."""
    cin = w.geo_out + (16 if w.view_dirs else 0)
    return 2 * (128 + ((cin + 128) if w.colour else 0))


def method_bytes_per_sample(w, precision, kernel):
    """Algorithmic bytes per sample of the METHOD (independent of this implementation's
    design): the hash-grid gather of S3 (8 corners x L levels x F features, 2 B each from the
    FP16 tables, 4 B from binary32 ones), the scatter of S7c (8 corners x L x F binary32
    gradient updates = 4 B each, counted once), and the per-sample streams the kernel must
    read or write (xyz 12 B in; sigma, rgb 16 B out for the forward; dsigma, drgb 16 B in for
    the backward).  The whole step adds both field kernels' figures minus the shared xyz
    read plus the compositing's t, delta (8 B)."""
    fb = 2 if precision != "fp32" else 4
    gather = w.L * 8 * w.F * fb
    scatter = w.L * 8 * w.F * 4
    if kernel == "field_forward":
        return gather + 12 + 16
    if kernel == "field_backward":
        return scatter + 12 + 16
    if kernel == "step":
        return gather + scatter + 12 + 8 + 16 + 16
    return None


def design_bytes_per_sample(w, precision, kernel, saved):
    """Bytes per sample this implementation moves beyond the method's (its design choices):
    the forward's feature store for the backward (split FP16, or high parts only with stored
    activations), the stored activations, and their reads in the backward."""
    if precision == "fp32":
        return 0
    IN = max(16, w.L * w.F)
    feat = 2 * IN if saved else 4 * IN
    acts = act_bytes_per_sample(w) if saved else 0
    if kernel in ("field_forward", "field_backward"):
        return feat + acts + (16 if (saved and kernel == "field_backward") else 0)
    return None


def field_backward_work(w, precision, saved=False):
    """Algorithmic FLOPs and HBM bytes per sample of the fused field backward.
    FLOPs: the recomputed MLP forward (unless the forward stored its activations,
    `saved`) + input gradients + weight gradients (3 or 2 x the forward MACs x 2).
    HBM bytes: the binary32 path re-gathers the 8 corners of L levels x F
    binary32 table entries (the tables and their gradients are L2-resident, so
    the gather is counted once as a stream here only for the binary32 baseline);
    the mixed path reads back its stored features (split FP16, 4 B x L*F; the
    E4M3 path its 1-byte codes), or with stored activations their high parts
    (2 B x L*F) and the activations, plus (sigma, rgb) (16 B); all read xyz
    (12 B) and the upstream gradient (16 B).
    The scatter-add of the table gradient (8 corners x L x F binary32 RMW) goes
    to L2-resident memory and is reported as l2_red_bytes, not as HBM bytes.
    With view directions the first colour layer's input gradient covers the g
    columns only (the direction encoding has no parameters behind it), and each
    sample reads its ray index (4 B; the directions themselves are per ray)."""
    saved = saved and precision != "fp32"
    fl = (2 if saved else 3) * mlp_flops_per_sample(w) - (2 * 16 * 64 if w.view_dirs else 0)
    vd = 4 if w.view_dirs else 0
    if precision == "fp32":
        feat = w.L * 8 * w.F * 4
    elif precision == "mixed_e4m3":
        feat = max(16, w.L * w.F)       # the E4M3 codes, 1 B per feature
    elif saved:
        feat = 2 * max(16, w.L * w.F)   # high parts only
    else:
        feat = 4 * max(16, w.L * w.F)
    if saved:
        feat += act_bytes_per_sample(w) + 16
    return fl, feat + 12 + 16 + vd


def field_forward_work(w, precision, saved=False):
    """FLOPs: the MLP forward.  HBM bytes: xyz in (12 B), (sigma, rgb) out
    (16 B) and, on the mixed path, the split-FP16 features written for the
    backward (4 B x L*F) and, with `saved`, the stored activations; the table
    gather (8 corners x L x F) hits the L2-resident tables and is reported as
    l2_gather_bytes."""
    vd = 4 if w.view_dirs else 0  # the sample's ray index (view-direction colour input)
    if saved and precision == "mixed":
        vd += act_bytes_per_sample(w) - 2 * max(16, w.L * w.F)  # activations stored; feature low parts not
    if precision == "fp32":
        return mlp_flops_per_sample(w), 12 + 16 + vd
    if precision == "mixed_e4m3":
        # gather pass: xyz in, binary32 features out; MLP pass: features in, codes and (sigma, rgb) out
        IN = w.L * w.F
        return mlp_flops_per_sample(w), 12 + 4 * IN + 4 * IN + max(16, IN) + 16
    return mlp_flops_per_sample(w), 12 + 16 + 4 * max(16, w.L * w.F) + vd


# DRAM bytes per sample (ncu dram__bytes_read.sum + dram__bytes_write.sum over the samples of the
# launch) of each field kernel, keyed by (precision, kernel, stored activations, forward shape:
# "split" = dedicated gather warps, "chain" = every thread gathers then runs the chain), with the
# capture it comes from.  Traffic grows with the samples processed, so a launch's traffic is this
# figure x its samples.  Only kernels unchanged since their capture have an entry: the others report
# traffic null.
WINDOW_CAPTURE = "window2x2_full, 65536 rays (7.98 M samples)"
TILE_CAPTURE = "tile512_full, 32768 rays (2.86 M samples)"
MEASURED_DRAM_PER_SAMPLE = {("mixed", "field_forward", True, "split"): (702.4, WINDOW_CAPTURE),
                            ("mixed", "field_backward", True, ""): (787.7, WINDOW_CAPTURE),
                            ("fp32", "field_backward", False, ""): (736.6, TILE_CAPTURE),
                            ("fp32", "field_forward", False, ""): (42.5, TILE_CAPTURE)}


def dram_capture(prec_key, kernel, saved, split):
    """(measured DRAM bytes per sample, capture) of a field kernel in the given configuration, or
    None (no capture of that kernel as it stands)."""
    shape = ("split" if split else "chain") if (kernel == "field_forward" and prec_key == "mixed") else ""
    return MEASURED_DRAM_PER_SAMPLE.get((prec_key, kernel, bool(saved), shape))


def dram_bytes_per_sample(prec_key, kernel, saved, split):
    """Measured DRAM bytes per sample of a field kernel in the given configuration, or None."""
    c = dram_capture(prec_key, kernel, saved, split)
    return c[0] if c else None


# ---- clocks -------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- reference arm / CPU baseline: the FP64 oracle ------------------------------
def oracle_sample(w, cams, targets, params, seed, n_rays):
    """Time one oracle training step on n_rays rays of the workload; returns
    (samples, seconds)."""
    from oracle import step as OS
    cfg = OS.ModelConfig(L=w.L, F=w.F, log2_T=w.log2_T, n_min=w.n_min, n_max=w.n_max, hidden=64,
                         geo_out=w.geo_out, colour=w.colour, shared_colour=w.shared_colour, n_slots=w.n_slots,
                         K_ray=w.K_ray, K_min=w.K_min, K_max=w.K_max, first_layer=w.first_layer,
                         view_dirs=w.view_dirs)
    pix = W.batch(w, cams, 1000 + seed, n_rays=n_rays)
    flat = params.astype(np.float64)
    n = len(flat)
    t0 = time.perf_counter()
    res = OS.train_step(cfg, flat, np.zeros(n), np.zeros(n), [0] * cfg.n_optimisers(), cams, w.window(), pix,
                        targets, seed, 0)
    dt = time.perf_counter() - t0
    return int(res.seg.ray_off[-1]), dt


def cpu_model():
    """The host CPU's model name (/proc/cpuinfo), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads", 1) for d in threadpool_info()]
        return max(n) if n else 1
    except Exception:
        return 1


def make_inputs(w, n_grid_params):
    """Cameras, target images and initial parameters of the workload;
    n_grid_params = table parameters per tile (from the caller's layout)."""
    cams = W.cameras(w)
    targets = synth.smooth_images(w.seed + 17, w.n_views, w.px, w.px)
    geo = [(64, w.L * w.F), (64, 64), (w.geo_out, 64)]
    col = [(64, w.geo_out + (16 if w.view_dirs else 0)), (64, 64), (3, 64)] if w.colour else []
    n_col = (1 if w.shared_colour else w.n_slots) if w.colour else 0
    params = W.init_params(n_grid_params, geo, col, w.n_slots, n_col, w.seed)
    return cams, targets, params


def oracle_grid_params(w):
    from oracle import hashgrid
    return hashgrid.layout(w.L, w.F, w.log2_T, w.n_min, w.n_max).n_params


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cams, targets, params = make_inputs(w, oracle_grid_params(w))
    tot_s = tot_t = 0.0
    for i in range(args.warmup):
        oracle_sample(w, cams, targets, params, i, min(32, args.cpu_rays))
    for i in range(args.steps):
        s, t = oracle_sample(w, cams, targets, params, 100 + i, args.cpu_rays)
        tot_s += s
        tot_t += t
    v = tot_s / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "rays_per_step": args.cpu_rays, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": "%d oracle steps of %d rays of %s" % (args.steps, args.cpu_rays, w.name),
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- our arm ------------------------------------------------------------------------
def reduce_over_ranks(maxes, sums, device):
    """Whole-job figures of independent replicas: the max over ranks of each time,
    the sum over ranks of each count (torch.distributed must be initialised)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(maxes, device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor(sums, device=device, dtype=torch.float64)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(x) for x in t], [float(x) for x in c]


def time_steps(torch, tr, batches, steps, stream):
    """Device time (ms) and samples of `steps` eager training steps."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    counts = []
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(steps):
        tr.train_step(batches[i % len(batches)], stream=stream)
        counts.append(tr.state[3:4].clone())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), int(sum(int(c.item()) & 0xFFFFFFFF for c in counts))


def time_graph(torch, tr, batches, steps):
    """Capture one training step into a CUDA graph (static pixel buffer) and time
    `steps` replays, each preceded by a device copy of that step's batch."""
    static_pix = torch.empty_like(batches[0])
    static_pix.copy_(batches[0])
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        tr.train_step(static_pix, stream=side)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        tr.train_step(static_pix, stream=torch.cuda.current_stream())
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    counts = []
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(steps):
        static_pix.copy_(batches[i % len(batches)], non_blocking=True)
        g.replay()
        counts.append(tr.state[3:4].clone())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), int(sum(int(c.item()) & 0xFFFFFFFF for c in counts))


def reduction_probe(torch, snk, ctx, n_entries, reps=3):
    """Peak of the reduction roofline: the library's stand-alone reduction probe
    (snk_l2_reduction_probe: nothing but fire-and-forget float reductions to random 16-byte
    slots, full occupancy) on a table of one tile's gradient size (n_entries float2 entries),
    timed with CUDA events after a warm-up.  Returns operations (= L2 sectors touched) per
    second for 16-byte (v4) and 8-byte (v2) reductions."""
    n16 = max(1, (int(n_entries) * 8) // 16)
    table = torch.zeros(n16 * 4, dtype=torch.float32, device="cuda")
    n_ops = 1 << 29
    out = {"table_bytes": n16 * 16, "ops_per_call": n_ops}
    for width in (16, 8):
        ctx.call("snk_l2_reduction_probe", snk.ptr(table), n16, n_ops, width, 1, None)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for r in range(reps):
            ctx.call("snk_l2_reduction_probe", snk.ptr(table), n16, n_ops, width, 2 + r, None)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out["v4" if width == 16 else "v2"] = {"ms": ms, "ops_per_s": n_ops / ms * 1e3}
    del table
    torch.cuda.empty_cache()
    return out


# Table-gradient reductions per sample of the fused backward: ncu lts__t_sectors_srcunit_tex_op_red.sum
# (each reduction an SM issues, counted once: one 16- or 8-byte reduction is one sector operation;
# lts__t_sectors_op_red also counts the half of them that cross to the other die's L2 a second time)
# over the samples of the launch, keyed by (precision, stored activations), with the capture.  The
# probe's rate is in the same unit.  A kernel changed since its capture has no entry.
MEASURED_RED_SECTORS_PER_SAMPLE = {("mixed", True): (69.4, WINDOW_CAPTURE)}

# Table-gather sectors per sample of the forward with dedicated gather warps: ncu
# l1tex__t_sectors_pipe_lsu_mem_global_op_ld.sum (requested from L1) and
# lts__t_sectors_srcunit_tex_op_read.sum (reaching L2: L1 misses and the streams) over the samples,
# keyed by (precision, stored activations, split forward), with the capture.  The method's own
# gather is 8 corners x L x F FP16 = 512 B a sample, 16 sectors if every corner pair shared one.
GATHER_CAPTURE = "window2x2_full, 16384 rays (1.99 M samples), --set full"
MEASURED_GATHER_SECTORS_PER_SAMPLE = {("mixed", True, 1): (65.3, 45.6, GATHER_CAPTURE)}


def roofline_of(w, prec_key, name, per_launch_s, units, saved, split, pk, probe=None):
    """The dominant kernel's roofline: achieved = the method's algorithmic bytes per sample x
    the samples of one launch / the launch's CUDA-event time, against the measured HBM peak;
    beside it the tensor-pipe figure, the bytes this implementation adds by design, and (field
    backward) the L2 reduction roofline against the probe's measured rate."""
    method = method_bytes_per_sample(w, prec_key, name)
    if method is None:
        return {"kernel": name, "bound": "unknown", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}
    gbs = method * units / per_launch_s / 1e9
    dram = dram_bytes_per_sample(prec_key, name, saved, split)
    cap = dram_capture(prec_key, name, saved, split)
    roof = {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / pk["hbm_gbs"], "traffic": dram * units if dram is not None else None,
            "traffic_source": ("ncu DRAM bytes per sample of the %s capture x samples per launch" % cap[1]) if cap
            else "no capture of this kernel as it stands",
            "peak_source": "%s hbm_gbs" % pk["source"], "algorithmic_bytes_per_sample": method,
            "units_per_launch": units, "launch_ms": per_launch_s * 1e3}
    design = design_bytes_per_sample(w, prec_key, name, saved)
    if design:
        roof["design_bytes_per_sample"] = design
        roof["achieved_with_design_bytes"] = (method + design) * units / per_launch_s / 1e9
    fl = (field_backward_work if name == "field_backward" else field_forward_work)(w, prec_key, saved)[0]
    if prec_key == "fp32":
        peak = 148 * 128 * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        roof["alu"] = {"achieved": fl * units / per_launch_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                       "frac": fl * units / per_launch_s / 1e12 / peak,
                       "peak_source": "148 SMs x 128 FP32 lanes x 2 FLOP x max SM clock (derived)"}
    else:
        tfl = fl * units / per_launch_s / 1e12
        roof["tensor"] = {"achieved": tfl, "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                          "frac": tfl / pk["bf16_tflops_sustained"],
                          "peak_source": "%s bf16_tflops_sustained (FP16 dense rate = BF16 rate)" % pk["source"]}
    red = MEASURED_RED_SECTORS_PER_SAMPLE.get((prec_key, bool(saved)))
    if name == "field_backward" and red is not None and probe:
        sec = red[0] * units / per_launch_s
        pv = probe["v4"]["ops_per_s"]
        roof["l2_reduction"] = {"bound": "l2_red", "achieved": sec / 1e9, "peak": pv / 1e9, "unit": "G sectors/s",
                                "frac": sec / pv, "sectors_per_sample": red[0],
                                "peak_source": "snk_l2_reduction_probe, 16-byte reductions, measured in this run",
                                "sectors_source": "ncu lts__t_sectors_srcunit_tex_op_red.sum per sample, %s" % red[1]}
    return roof


def run_ours(args, w):
    import torch
    import torch.distributed as dist
    from paper_2507_01631_b300 import snk, build as B
    from paper_2507_01631_b300.trainer import Trainer, model_from_workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    if args.precision == "mixed":
        precision = snk.SNK_MIXED_E4M3 if w.first_layer == "e4m3" else snk.SNK_MIXED
    else:
        precision = snk.SNK_FP32
    prec_key = {snk.SNK_FP32: "fp32", snk.SNK_MIXED: "mixed", snk.SNK_MIXED_E4M3: "mixed_e4m3"}[precision]
    model = model_from_workload(w, precision)
    cams, targets, params = make_inputs(w, snk.layout(model).grid_params)
    ctx = snk.Context(local)
    crops = [torch.from_numpy(t).cuda() for t in targets]
    ctx.set_views(cams, crops)
    mode = {"segments": snk.SNK_SAMPLE_SEGMENTS, "uniform": snk.SNK_SAMPLE_UNIFORM,
            "points": snk.SNK_SAMPLE_POINTS}[args.sampler_mode]
    sampler = snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 1234 + rank, 0, mode=mode)
    tr = Trainer(ctx, model, snk.window_struct(w.window()), sampler, params)
    batches_h = [W.batch(w, cams, 50 + i + 1000 * rank).view(np.int32) for i in range(N_BATCHES)]
    batches = [torch.from_numpy(b).cuda() for b in batches_h]
    nseg = 1 + (w.nx == 2) + (w.ny == 2)
    ctx.reserve(w.n_rays, ctx.max_samples(snk.window_struct(w.window()), sampler, w.n_rays))
    stream = torch.cuda.current_stream()

    # launch shapes: picked on the first batch, outside the timed region
    tuning = tr.autotune(batches[0], stream=stream) if args.autotune else ctx.tuning()
    if args.bwd_saved != "auto":
        # the forward shape the tuner picked for the other mode may differ; keep its choice otherwise
        ctx.set_tuning(tc_bwd_saved=int(args.bwd_saved))
        tuning = ctx.tuning()
    if args.fwd_split != "auto":
        ctx.set_tuning(tc_fwd_split=int(args.fwd_split))
        tuning = ctx.tuning()
    # warm-up
    for i in range(args.warmup):
        tr.train_step(batches[i % N_BATCHES], stream=stream)
    rc = ctx.sync_status(tr.state)
    if rc not in (snk.SNK_OK, snk.SNK_ERR_OVERFLOW):
        raise RuntimeError("warm-up failed with status %d: %s" % (rc, ctx.lib.snk_last_error(ctx.h)))

    # timed region (device-resident inputs)
    samples = []
    clock = ClockSampler(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if args.stage_timing:
        ctx.stage_timing(True)
    launches0 = ctx.lib.snk_launch_count()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clock.start()
    time.sleep(0.3)
    ev0.record(stream)
    n_state = []
    for i in range(args.steps):
        tr.train_step(batches[i % N_BATCHES], stream=stream)
        n_state.append(tr.state[3:4].clone())  # n_samples of this step (device copy, no sync)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clock.stop()
    launches = ctx.lib.snk_launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    stages = ctx.stage_times() if args.stage_timing else {}
    if args.stage_timing:
        ctx.stage_timing(False)
    n_samples = int(sum(int(x.view(torch.int32).item()) & 0xFFFFFFFF for x in n_state))
    st = tr.read_state()
    rc = ctx.sync_status(tr.state)

    # end to end through host buffers: pinned pixels in, loss + counts out
    pin_in = [torch.from_numpy(b).pin_memory() for b in batches_h]
    pix_dev = torch.empty_like(batches[0])
    state_host = torch.empty(snk.STATE_WORDS, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_samples = 0
    for i in range(args.steps):
        pix_dev.copy_(pin_in[i % N_BATCHES], non_blocking=True)
        tr.train_step(pix_dev, stream=stream)
        state_host.copy_(tr.state, non_blocking=True)
        stream.synchronize()
        e2e_samples += int(state_host[3].item()) & 0xFFFFFFFF
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    extra = {}
    if args.graph:
        gms, gs = time_graph(torch, tr, batches, args.steps)
        extra["graph_replay"] = {"value": gs / (gms / 1000.0), "unit": "samples/s", "ms_per_step": gms / args.steps,
                                 "steps": args.steps}
    probe = None
    if args.red_ceiling:
        probe = reduction_probe(torch, snk, ctx, snk.layout(model).n_entries)
        extra["l2_reduction_probe"] = probe
    if args.compare_fp32 and args.precision == "mixed":
        m32 = model_from_workload(w, snk.SNK_FP32)
        tr32 = Trainer(ctx, m32, snk.window_struct(w.window()), sampler, params)
        if args.autotune:
            tr32.autotune(batches[0], stream=stream)
        tr32.train_step(batches[0], stream=stream)
        ctx.stage_timing(True)
        fms, fs = time_steps(torch, tr32, batches, args.fp32_steps, stream)
        st32 = ctx.stage_times()
        ctx.stage_timing(False)
        rc32 = ctx.sync_status(tr32.state)
        # its own roofline: the dominant stage (a per-tile field launch chain) against the
        # binary32 ALU peak and, for the backward, the reduction probe
        nm32, (ms32, calls32) = max(st32.items(), key=lambda kv: kv[1][0])
        per32 = fs / args.fp32_steps
        roof32 = roofline_of(w, "fp32", nm32, ms32 / max(calls32, 1) / 1000.0, per32, False, 0, peaks(), None)
        extra["fp32_per_tile"] = {"value": fs / (fms / 1000.0), "unit": "samples/s",
                                  "ms_per_step": fms / args.fp32_steps, "steps": args.fp32_steps, "status": rc32,
                                  "launches": "one field launch per tile and direction, eager",
                                  "stage_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in st32.items()},
                                  "roofline": roof32}
        del tr32

    t_max = ms
    tot_samples = n_samples
    e2e_tot = e2e_samples
    e2e_max = e2e_ms
    if world > 1:
        (t_max, e2e_max), (tot_samples, e2e_tot) = reduce_over_ranks([ms, e2e_ms], [n_samples, e2e_samples], "cuda")
    value = tot_samples / (t_max / 1000.0)
    e2e_value = e2e_tot / (e2e_max / 1000.0)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # roofline of the dominant stage
    pk = peaks()
    roof = None
    if stages:
        name, (sms, calls) = max(stages.items(), key=lambda kv: kv[1][0])
        per_launch_s = (sms / max(calls, 1)) / 1000.0
        per_step_samples = n_samples / max(args.steps, 1)
        saved = bool(tuning.get("tc_bwd_saved", 0)) and prec_key != "fp32"
        if saved and st.get("bwd_mode") == 2:
            saved = False  # the step fell back to recomputing its activations
        roof = roofline_of(w, prec_key, name, per_launch_s, per_step_samples, saved, tuning.get("tc_fwd_split", 0),
                           pk, probe)
        step_bytes = method_bytes_per_sample(w, prec_key, "step")
        step_s = (t_max / args.steps) / 1000.0
        roof["step"] = {"algorithmic_bytes_per_sample": step_bytes,
                        "achieved": step_bytes * per_step_samples / step_s / 1e9, "unit": "GB/s",
                        "frac": step_bytes * per_step_samples / step_s / 1e9 / pk["hbm_gbs"]}
        roof["stage_ms_per_step"] = {k: v[0] / max(v[1], 1) for k, v in stages.items()}
        if name != "field_forward" and "field_forward" in stages:
            # the second field kernel beside the dominant one, with its gather sectors
            fs, fc = stages["field_forward"]
            split = tuning.get("tc_fwd_split", 0)
            fwd = roofline_of(w, prec_key, "field_forward", (fs / max(fc, 1)) / 1000.0, per_step_samples, saved,
                              split, pk, None)
            g = MEASURED_GATHER_SECTORS_PER_SAMPLE.get((prec_key, bool(saved), int(split)))
            if g is not None:
                fwd["gather_sectors_per_sample"] = {"l1_requested": g[0], "l2_read": g[1], "method": 16,
                                                    "source": "ncu, %s" % g[2]}
            roof["field_forward"] = fwd

    cpu = None
    if not args.no_cpu_baseline:
        from synth import workloads as W2  # noqa: F401
        tot_s = tot_t = 0.0
        for i in range(2):
            s, t = oracle_sample(w, cams, targets, params, 200 + i, args.cpu_rays)
            tot_s += s
            tot_t += t
        cpu = {"value": tot_s / tot_t, "unit": "samples/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": "2 oracle steps of %d rays of %s (%d samples), FP64 numpy" % (args.cpu_rays, w.name,
                                                                                     int(tot_s)),
               "nproc": os.cpu_count(), "cpu_model": cpu_model()}
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "mixed": "f16 (split) / f32 acc",
                                       "mixed_e4m3": "e4m3 first layer, f16 (split) / f32 acc"}[prec_key],
        "data": "synthetic",
        "config": {"workload": w.name, "precision": prec_key, "rays_per_step": w.n_rays,
                   "samples_per_step": n_samples / args.steps, "tiles": w.n_slots,
                   "grid": "L%d F%d T2^%d N%d-%d" % (w.L, w.F, w.log2_T, w.n_min, w.n_max),
                   "views": "%d x %dpx %s" % (w.n_views, w.px, "rpc3" if w.cam_kind else "affine"),
                   "parallelism": "replicas" if world > 1 else "single",
                   "launch_shapes": tuning,
                   **({"view_dirs": "SH degrees 0..3 of the ray direction"} if w.view_dirs else {}),
                   **({"sampler": args.sampler_mode} if args.sampler_mode != "segments" else {}),
                   "l2": "working set per step > L2 (sample buffers %.2f GB)" % (n_samples / args.steps * 52 / 1e9)},
        "rays_per_s": st["n_accepted"] * args.steps / (ms / 1000.0) * world,
        "final_loss": st["loss"], "status": rc,
        "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": int(batches_h[0].nbytes),
                "d2h_bytes_per_step": int(snk.STATE_WORDS * 4)},
        "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "cpu_baseline": cpu,
    }
    line.update(extra)
    if "fp32_per_tile" in extra and extra["fp32_per_tile"]["value"] > 0:
        line["speedup_vs_fp32_per_tile"] = (n_samples / (ms / 1000.0)) / extra["fp32_per_tile"]["value"]
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    over = {}
    if args.rays > 0:
        over["n_rays"] = args.rays
    if args.view_dirs:
        over["view_dirs"] = True
    w = W.get(args.workload, **over)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
