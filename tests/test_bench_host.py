"""Host logic of bench.py's roofline (CPU only): the method's algorithmic bytes counted by hand,
the roofline fields recomputed from them, measured DRAM figures present exactly for the kernels
captured as they stand, and those figures consistent with the bytes the kernels stream."""
import bench
from synth import workloads as W


def test_dram_figures_cover_the_default_configurations_only():
    # the benchmark's default shapes (stored activations, dedicated gather warps) and the binary32 arm
    assert bench.dram_bytes_per_sample("mixed", "field_forward", True, 1) is not None
    assert bench.dram_bytes_per_sample("mixed", "field_backward", True, 1) is not None
    for kernel in ("field_forward", "field_backward"):
        assert bench.dram_bytes_per_sample("fp32", kernel, False, 0) is not None
    # shapes whose kernels changed since their last capture, and the E4M3 kernels: traffic null
    assert bench.dram_bytes_per_sample("mixed", "field_forward", False, 0) is None
    assert bench.dram_bytes_per_sample("mixed", "field_backward", False, 1) is None
    assert bench.dram_bytes_per_sample("mixed_e4m3", "field_backward", True, 0) is None


def test_gather_sectors_cover_the_default_forward_only():
    # the default forward (stored activations, dedicated gather warps) has its capture; others none
    assert bench.MEASURED_GATHER_SECTORS_PER_SAMPLE.get(("mixed", True, 1)) is not None
    assert bench.MEASURED_GATHER_SECTORS_PER_SAMPLE.get(("mixed", True, 0)) is None
    assert bench.MEASURED_GATHER_SECTORS_PER_SAMPLE.get(("fp32", False, 0)) is None


def test_method_bytes_of_the_headline_workload_by_hand():
    """The method's algorithmic bytes per sample for L = 16 levels x F = 2 features: the gather
    reads 8 corners x 16 x 2 FP16 = 512 B (binary32 tables: 1024 B), the scatter adds 8 x 16 x 2
    binary32 = 1024 B; the field kernels' streams xyz 12 B in, (sigma, rgb) 16 B out (forward) or
    (dsigma, drgb) 16 B in (backward); the step 512 + 1024 + xyz 12 + t, delta 8 + 16 + 16 = 1588."""
    w = W.get("window2x2_full")
    assert bench.method_bytes_per_sample(w, "mixed", "field_forward") == 512 + 12 + 16
    assert bench.method_bytes_per_sample(w, "mixed", "field_backward") == 1024 + 12 + 16
    assert bench.method_bytes_per_sample(w, "fp32", "field_forward") == 1024 + 12 + 16
    assert bench.method_bytes_per_sample(w, "mixed", "step") == 1588
    # what the design adds: the stored activations (544 B) and feature high parts (64 B), read
    # back with (sigma, rgb) 16 B by the backward
    assert bench.design_bytes_per_sample(w, "mixed", "field_backward", True) == 544 + 64 + 16
    assert bench.design_bytes_per_sample(w, "mixed", "field_forward", False) == 128


def test_roofline_fields_recomputed_by_hand():
    """achieved = algorithmic bytes per sample x samples of the launch / launch time; frac =
    achieved / the measured peak; the reduction roofline divides the measured reductions per
    sample x samples / time by the probe's rate."""
    w = W.get("window2x2_full")
    pk = {"hbm_gbs": 6500.0, "bf16_tflops_sustained": 1400.0, "source": "test"}
    probe = {"v4": {"ops_per_s": 200e9}}
    units, t = 64e6, 0.035
    r = bench.roofline_of(w, "mixed", "field_backward", t, units, True, 1, pk, probe)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 1052 * units / t / 1e9) < 1e-9
    assert abs(r["frac"] - 1052 * units / t / 1e9 / 6500.0) < 1e-12
    red, _ = bench.MEASURED_RED_SECTORS_PER_SAMPLE[("mixed", True)]
    assert abs(r["l2_reduction"]["frac"] - red * units / t / 200e9) < 1e-12
    assert abs(r["traffic"] - bench.dram_bytes_per_sample("mixed", "field_backward", True, 1) * units) < 1.0
    assert abs(r["tensor"]["achieved"] - 2 * 2 * 12480 * units / t / 1e12) < 1e-9


def test_forward_roofline_fields_recomputed_by_hand():
    """The forward's entry: 540 method bytes a sample (512 B gather, xyz 12 B, (sigma, rgb) 16 B)
    x samples / launch time against the measured peak; its traffic from the forward's own capture;
    tensor FLOPs 2 x 12,480 a sample; no reduction roofline."""
    w = W.get("window2x2_full")
    pk = {"hbm_gbs": 6500.0, "bf16_tflops_sustained": 1400.0, "source": "test"}
    units, t = 64e6, 0.018
    r = bench.roofline_of(w, "mixed", "field_forward", t, units, True, 1, pk, {"v4": {"ops_per_s": 200e9}})
    assert r["bound"] == "hbm" and abs(r["achieved"] - 540 * units / t / 1e9) < 1e-9
    assert abs(r["frac"] - 540 * units / t / 1e9 / 6500.0) < 1e-12
    assert abs(r["traffic"] - bench.dram_bytes_per_sample("mixed", "field_forward", True, 1) * units) < 1.0
    assert abs(r["tensor"]["achieved"] - 2 * 12480 * units / t / 1e12) < 1e-9
    assert "l2_reduction" not in r


def test_algorithmic_work_of_the_headline_workload_by_hand():
    """The implementation's own per-sample work for the 2x2 window (L = 16 levels x F = 2
    features, 64-wide hidden layers, 16-d embedding, colour net), counted by hand from the layer
    sizes: MACs 32*64 + 64*64 + 64*16 (density) + 16*64 + 64*64 + 64*3 (colour) = 12,480;
    stored activations h1, h2, c1, c2 (64 FP16 each) + g (16 FP16) = 544 B; forward bytes xyz 12 +
    (sigma, rgb) 16 + features (FP16 high parts 64 B, or high and low 128 B when nothing else is
    stored) + the activations; backward bytes the same reads back plus the upstream gradient 16 B,
    FLOPs 2x the forward MACs x 2 (3x when recomputing)."""
    w = W.get("window2x2_full")
    assert bench.mlp_flops_per_sample(w) == 2 * 12480
    assert bench.act_bytes_per_sample(w) == 544
    assert bench.field_forward_work(w, "mixed", True) == (2 * 12480, 12 + 16 + 64 + 544)
    assert bench.field_forward_work(w, "mixed", False) == (2 * 12480, 12 + 16 + 128)
    assert bench.field_backward_work(w, "mixed", True) == (2 * 2 * 12480, 64 + 544 + 16 + 12 + 16)
    assert bench.field_backward_work(w, "mixed", False) == (3 * 2 * 12480, 128 + 12 + 16)
    # the binary32 baseline re-gathers 8 corners x 16 levels x 2 binary32 features
    assert bench.field_backward_work(w, "fp32", False) == (3 * 2 * 12480, 8 * 16 * 2 * 4 + 12 + 16)


def test_measured_traffic_is_close_to_the_streamed_bytes():
    """ncu's DRAM bytes per sample of the default kernels on the 2x2 window exceed the bytes they
    stream (activations, features, per-sample inputs and outputs) by at most 25 %: the excess is
    table and gradient lines that do not stay in L2 over a step of four tiles (their FP16 tables
    and cell copies ~34 MB a tile, binary32 gradients and cell gradients ~69 MB a tile, against
    126 MB of L2 shared with the streams); no kernel re-reads its own streams."""
    w = W.get("window2x2_full")
    for kernel, work in (("field_forward", bench.field_forward_work), ("field_backward", bench.field_backward_work)):
        measured = bench.dram_bytes_per_sample("mixed", kernel, True, 1)
        _, streamed = work(w, "mixed", True)
        assert 0.95 <= measured / streamed <= 1.25, (kernel, measured, streamed)
