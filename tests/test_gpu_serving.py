"""GPU tests of the continuous-batching serving loop.

Each job's result must be the same whether it is served alone or in a mix that
arrives, overlaps and leaves around it; admission respects the memory budget; every
job ends in a defined state and the report carries finite latency percentiles.
"""
import numpy as np
import pytest

import lbm_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def small_jobs(n, seed, rate_hz=200.0, dmin=12, dmax=28):
    from paper_0811_4593_gb300.serving import Job
    reqs = inp.serving_requests(n, seed, rate_hz, dmin, dmax)
    return [Job(r.rid, r.arrival_s, inp.request_workload(r)) for r in reqs], reqs


def test_every_job_finishes_with_a_report():
    from paper_0811_4593_gb300.serving import Server
    jobs, reqs = small_jobs(10, 3)
    srv = Server("f32", capacity=8, budget_bytes=4e9, round_steps=50, max_steps=1500, target=1e-6, plateau_checks=5)
    results, rep = srv.serve(jobs)
    assert [r.jid for r in results] == list(range(10))
    for r in results:
        assert r.status in ("converged", "plateau", "step_cap", "diverged")
        assert r.steps % 50 == 0 and 0 < r.steps <= 1500
        assert r.finished_s >= r.admitted_s >= r.arrival_s - 1e-9
        if r.status == "converged":
            assert r.residual < 1e-6
    assert rep["jobs"] == 10
    assert np.isfinite(rep["p50_time_to_steady_s"]) and np.isfinite(rep["p99_time_to_steady_s"])
    assert rep["p99_time_to_steady_s"] >= rep["p50_time_to_steady_s"]
    assert rep["aggregate_mlups"] > 0
    assert rep["peak_active"] <= 8


def test_job_result_is_the_same_alone_and_in_the_mix():
    from paper_0811_4593_gb300.serving import Job, Server
    jobs, _ = small_jobs(7, 11, rate_hz=400.0)
    kw = dict(capacity=4, budget_bytes=4e9, round_steps=40, max_steps=800, target=1e-7, plateau_checks=4,
              keep_populations=True)
    mixed, rep = Server("f32", **kw).serve(jobs)
    assert rep["peak_active"] >= 2  # the jobs really overlapped
    for probe in (0, 3, 6):
        alone, _ = Server("f32", **kw).serve([Job(probe, 0.0, jobs[probe].workload)])
        a, m = alone[0], mixed[probe]
        assert (a.steps, a.status) == (m.steps, m.status)
        assert a.history == m.history
        np.testing.assert_array_equal(a.populations, m.populations)


def test_admission_respects_the_memory_budget():
    from paper_0811_4593_gb300.serving import Job, Server, footprint_bytes
    wls = [inp.duct(24, 16, 16, 0.8, 0.04, 20.0) for _ in range(5)]
    one = footprint_bytes(24, 16, 16, "f32")
    jobs = [Job(i, 0.0, wl) for i, wl in enumerate(wls)]
    results, rep = Server("f32", capacity=8, budget_bytes=2.5 * one, round_steps=50, max_steps=200,
                          target=1e-12).serve(jobs, closed_loop=True)
    assert rep["peak_active"] == 2
    assert rep["peak_bytes"] <= 2.5 * one
    assert len(results) == 5
    with pytest.raises(ValueError):
        Server("f32", budget_bytes=one / 2).serve(jobs[:1])
