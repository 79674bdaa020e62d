"""Failure detection without a GPU fault: every mbarrier wait of the
tensor-core field kernels is bounded in time; when it gives up the kernel
sets the timeout bit of the step state and returns, the host reads
SNK_ERR_TIMEOUT, and the context stays usable.  The self-test entry point
runs that wait on an mbarrier that gets its arrival (completes) and on one
that never does (gives up after 2 s)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300 import build, snk
from paper_2507_01631_b300.trainer import Trainer, model_from_workload
from gpu_util import make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = snk.Context(0)
    yield c
    c.close()


def test_bounded_wait_completes_or_reports_a_timeout(ctx):
    state = torch.zeros(snk.STATE_WORDS, dtype=torch.int32, device="cuda")
    ctx.call("snk_wait_selftest", 1, snk.ptr(state), None)
    assert ctx.sync_status(state) == snk.SNK_OK
    t0 = time.time()
    ctx.call("snk_wait_selftest", 0, snk.ptr(state), None)
    assert ctx.sync_status(state) == snk.SNK_ERR_TIMEOUT
    assert 1.5 < time.time() - t0 < 60.0
    # the context and the device stay usable: a mixed training step on a fresh state succeeds
    case = make_case("tiny_window", n_rays=160, table_scale=0.3)
    w = case.w
    ctx.set_views(case.cams, [torch.from_numpy(t.astype(np.float32)).cuda() for t in case.targets])
    tr = Trainer(ctx, model_from_workload(w, snk.SNK_MIXED), snk.window_struct(w.window()),
                 snk.sampler_struct(w.K_ray, w.K_min, w.K_max, 0, 5, 0), case.params)
    tr.train_step(torch.from_numpy(case.pix.view(np.int32)).cuda())
    assert ctx.sync_status(tr.state) == snk.SNK_OK
    assert np.isfinite(tr.read_state()["loss"])
