"""Failure detection of the row-staged binary16 sweep, without a GPU fault.

The sweep waits on the bulk copies that stage population rows in shared memory with a
time limit of about one second. A test hook makes one CTA announce the copies of one
row group without issuing them, so that its waits run out: the kernel must end by
itself, flag the context's device error word, and the next synchronising call must
report it; afterwards the context must work normally again.
"""
import numpy as np
import pytest

import lbm_inputs as inp
from lbm_testlib import encode, noisy_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def test_a_stage_wait_that_runs_out_is_reported_and_the_context_recovers():
    import time

    import paper_0811_4593_gb300 as lbm
    from paper_0811_4593_gb300._binding import check
    wl = inp.channel(256, 6, 5, 0.7, (0.04, 0.01, 0.0))   # 256-node rows: the row-staged sweep
    s0 = encode(noisy_state((19, wl.nz, wl.ny, wl.nx), 5, u=(0.01, -0.004, 0.006)), "f16")
    with lbm.Lattice.from_workload(wl, "f16") as lat, lbm.Lattice.from_workload(wl, "f16") as ref:
        lat.set_populations(s0)
        check(lbm.lib().lbm_debug_drop_staged_copies(lat.ctx, 1), lat.ctx)
        t0 = time.perf_counter()
        lat.step(1)
        with pytest.raises(lbm.LBMError, match="gave up waiting"):
            lat.sync()
        waited = time.perf_counter() - t0
        assert 0.5 < waited < 30.0, waited          # the bounded waits ran out, then the kernel ended
        lat.sync()                                  # the error word was cleared by the report
        check(lbm.lib().lbm_debug_drop_staged_copies(lat.ctx, 0), lat.ctx)
        lat.set_populations(s0)
        lat.step(3)
        ref.set_populations(s0)
        ref.step(3)
        np.testing.assert_array_equal(lat.get_populations(), ref.get_populations())
