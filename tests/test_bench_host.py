"""Host logic of bench.py's roofline (CPU only): the measured DRAM bytes per sample exist for
every field kernel, backward mode and forward shape the benchmark can report, and for no
configuration without a capture."""
import bench


def test_dram_figures_cover_every_reported_configuration():
    for saved in (True, False):
        for split in (0, 1):
            assert bench.dram_bytes_per_sample("mixed", "field_forward", saved, split) is not None
        assert bench.dram_bytes_per_sample("mixed", "field_backward", saved, 1) is not None
    # the binary32 path stores nothing for its backward and has one forward shape
    for kernel in ("field_forward", "field_backward"):
        assert bench.dram_bytes_per_sample("fp32", kernel, False, 0) is not None
    # E4M3 kernels were not captured: traffic is reported as null
    assert bench.dram_bytes_per_sample("mixed_e4m3", "field_backward", True, 0) is None


def test_stored_activations_add_their_bytes():
    """Storing the activations adds their 544 B a sample of FP16 high parts and drops the
    features' 64 B of low parts (the backward then needs the high parts only): about 480 B more
    DRAM traffic a sample in the forward (written) and in the backward (read back)."""
    for kernel in ("field_forward", "field_backward"):
        extra = (bench.dram_bytes_per_sample("mixed", kernel, True, 1)
                 - bench.dram_bytes_per_sample("mixed", kernel, False, 1))
        assert 544 - 64 - 16 < extra < 544 - 64 + 32, (kernel, extra)


def test_algorithmic_work_of_the_headline_workload_by_hand():
    """The roofline numerators for the 2x2 window (L = 16 levels x F = 2 features, 64-wide
    hidden layers, 16-d embedding, colour net), counted by hand from the layer sizes:
    MACs 32*64 + 64*64 + 64*16 (density) + 16*64 + 64*64 + 64*3 (colour) = 12,480;
    stored activations h1, h2, c1, c2 (64 FP16 each) + g (16 FP16) = 544 B;
    forward bytes xyz 12 + (sigma, rgb) 16 + features (FP16 high parts 64 B, or high and low
    128 B when nothing else is stored) + the activations; backward bytes the same reads back
    plus the upstream gradient 16 B, FLOPs 2x the forward MACs x 2 (3x when recomputing)."""
    from synth import workloads as W
    w = W.get("window2x2_full")
    assert bench.mlp_flops_per_sample(w) == 2 * 12480
    assert bench.act_bytes_per_sample(w) == 544
    assert bench.field_forward_work(w, "mixed", True) == (2 * 12480, 12 + 16 + 64 + 544)
    assert bench.field_forward_work(w, "mixed", False) == (2 * 12480, 12 + 16 + 128)
    assert bench.field_backward_work(w, "mixed", True) == (2 * 2 * 12480, 64 + 544 + 16 + 12 + 16)
    assert bench.field_backward_work(w, "mixed", False) == (3 * 2 * 12480, 128 + 12 + 16)
    # the binary32 baseline re-gathers 8 corners x 16 levels x 2 binary32 features
    assert bench.field_backward_work(w, "fp32", False) == (3 * 2 * 12480, 8 * 16 * 2 * 4 + 12 + 16)


def test_measured_traffic_is_close_to_the_algorithmic_bytes():
    """ncu's DRAM bytes per sample stay within -10 % / +15 % of the algorithmic count: no
    kernel re-reads what it already moved (reads below the count hit lines still in L2)."""
    from synth import workloads as W
    w = W.get("window2x2_full")
    for kernel, work in (("field_forward", bench.field_forward_work), ("field_backward", bench.field_backward_work)):
        for saved in (True, False):
            measured = bench.dram_bytes_per_sample("mixed", kernel, saved, 1)
            _, algorithmic = work(w, "mixed", saved)
            assert 0.90 <= measured / algorithmic <= 1.15, (kernel, saved, measured, algorithmic)
