"""The reduction-rate probe (the peak of the scatter's roofline) does the work it claims:
n_ops reductions of width bytes of 1.0 to slots inside the table, spread over the whole
table, and nothing else (the table's sum grows by exactly n_ops x width / 4)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width", [16, 8])
def test_probe_adds_exactly_its_reductions(width):
    build.build()
    assert torch.cuda.is_available()
    ctx = snk.Context(0)
    try:
        n16 = 1_000_003  # not a power of two: the scaling onto [0, n16) must stay inside
        guard = 64
        buf = torch.zeros((n16 + guard) * 4, dtype=torch.float32, device="cuda")
        n_ops = 20_000_000
        ctx.call("snk_l2_reduction_probe", snk.ptr(buf), n16, n_ops, width, 7, None)
        torch.cuda.synchronize()
        t = buf.double().cpu().numpy()
        assert np.all(t[n16 * 4:] == 0.0), "write beyond the table"
        body = t[:n16 * 4].reshape(n16, 4)
        assert t.sum() == n_ops * width / 4
        assert np.all(body == np.round(body)) and body.min() >= 0
        per_slot = body.sum(1) / (width / 4)
        mean = n_ops / n16
        # uniform spread: every slot near the mean count (Poisson, 20 ops a slot on average)
        assert per_slot.max() < mean + 12 * np.sqrt(mean) + 10 and (per_slot == 0).mean() < 1e-3
        if width == 8:
            # each operation covers one half of its slot: both halves used about equally
            halves = body[:, :2].sum(), body[:, 2:].sum()
            assert abs(halves[0] - halves[1]) < 0.01 * sum(halves)
        # refused arguments
        for bad in [(snk.ptr(buf) + 4, n16, 1, width), (snk.ptr(buf), 0, 1, width), (snk.ptr(buf), n16, 1, 12)]:
            rc = ctx.lib.snk_l2_reduction_probe(ctx.h, bad[0], bad[1], bad[2], bad[3], 0, None)
            assert rc == snk.SNK_ERR_INVALID_ARG
    finally:
        ctx.close()
