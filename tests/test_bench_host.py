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
