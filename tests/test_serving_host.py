"""Host-side tests of the serving loop's scheduling (no GPU): admission by free slot
and memory budget in arrival order, retirement on convergence / plateau / step cap /
divergence, and the report's percentiles. A scripted batch stands in for the device:
each job's workload carries the residual it reports after every round."""
from dataclasses import dataclass, field

import pytest

from paper_0811_4593_gb300.serving import Job, Server, footprint_bytes, percentile


@dataclass
class Script:
    nx: int
    ny: int
    nz: int
    residuals: list            # residual reported after round 1, 2, ...; the last repeats
    diverge_at: int = 0        # round after which the status is "diverged" (0: never)


class FakeLattice:
    def __init__(self, wl):
        self.wl = wl
        self.closed = False
        self.rounds = 0

    @property
    def cells(self):
        return self.wl.nx * self.wl.ny * self.wl.nz

    def get_populations(self):
        return ("state", self.rounds)

    def close(self):
        self.closed = True


@dataclass
class FakeBatch:
    capacity: int
    precision: str
    slots: dict = field(default_factory=dict)
    log: list = field(default_factory=list)

    def free_slots(self):
        return [i for i in range(self.capacity) if i not in self.slots]

    def attach(self, slot, lat):
        assert slot not in self.slots
        self.slots[slot] = lat
        self.log.append(("attach", slot, lat.wl))

    def detach(self, slot):
        self.log.append(("detach", slot, self.slots.pop(slot).wl))

    def step(self, n, residual=False):
        assert residual
        for lat in self.slots.values():
            lat.rounds += 1

    def results(self):
        out = [(float("nan"), float("nan"), 1)] * self.capacity
        for slot, lat in self.slots.items():
            s = lat.wl
            r = s.residuals[min(lat.rounds, len(s.residuals)) - 1]
            st = -4 if s.diverge_at and lat.rounds >= s.diverge_at else 0
            out[slot] = (r, 1.0, st)
        return out

    def close(self):
        pass


class Clock:
    """Advances by `dt` per reading: deterministic arrival and latency arithmetic."""

    def __init__(self, dt=0.01):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def server(**kw):
    batches = []

    def make_batch(capacity, precision):
        batches.append(FakeBatch(capacity, precision))
        return batches[-1]

    kw.setdefault("round_steps", 100)
    srv = Server("f32", batch_factory=make_batch, lattice_factory=lambda wl, p, s: FakeLattice(wl), **kw)
    return srv, batches


def test_retirement_statuses():
    jobs = [
        Job(0, 0.0, Script(8, 8, 8, [1e-3, 1e-5, 1e-9])),                  # converges in round 3
        Job(1, 0.0, Script(8, 8, 8, [1e-3, 1e-6] + [2e-6] * 20)),          # plateau below the ceiling
        Job(2, 0.0, Script(8, 8, 8, [1e-2] * 40)),                         # never below the ceiling: cap
        Job(3, 0.0, Script(8, 8, 8, [1e-3] * 10, diverge_at=2)),           # diverges in round 2
    ]
    srv, _ = server(capacity=4, budget_bytes=1e12, max_steps=2000, target=1e-8, plateau_checks=5,
                    plateau_ceiling=1e-5)
    results, rep = srv.serve(jobs, closed_loop=True, clock=Clock())
    got = {r.jid: (r.status, r.steps) for r in results}
    assert got[0] == ("converged", 300)
    assert got[1] == ("plateau", 700)     # best at round 2, then 5 rounds without a new best
    assert got[2] == ("step_cap", 2000)
    assert got[3] == ("diverged", 200)
    assert rep["status_counts"] == {"converged": 1, "plateau": 1, "step_cap": 1, "diverged": 1}
    assert rep["jobs"] == 4 and rep["rounds"] == 20


def test_admission_by_slot_budget_and_arrival_order():
    one = footprint_bytes(16, 16, 16, "f32")
    jobs = [Job(i, 0.0, Script(16, 16, 16, [1e-9])) for i in range(7)]   # each done in one round
    srv, batches = server(capacity=3, budget_bytes=2.5 * one)
    results, rep = srv.serve(jobs, closed_loop=True, clock=Clock())
    assert rep["peak_active"] == 2                # the budget, not the 3 slots, binds
    assert rep["peak_bytes"] <= 2.5 * one
    attached = [e[2] for e in batches[0].log if e[0] == "attach"]
    assert attached == [j.workload for j in jobs]  # first in, first admitted
    admitted = [r.admitted_s for r in sorted(results, key=lambda r: r.jid)]
    assert admitted == sorted(admitted)
    with pytest.raises(ValueError):
        server(capacity=3, budget_bytes=one / 2)[0].serve(jobs[:1], closed_loop=True, clock=Clock())


def test_open_loop_waits_for_arrivals_and_measures_from_arrival():
    jobs = [Job(0, 0.0, Script(8, 8, 8, [1e-9])), Job(1, 5.0, Script(8, 8, 8, [1e-3, 1e-9]))]
    srv, _ = server(capacity=2, budget_bytes=1e12)
    results, rep = srv.serve(jobs, clock=Clock(0.5), idle_sleep=0.0)
    r0, r1 = results
    assert r1.admitted_s >= 5.0                    # not admitted before it arrived
    assert r1.finished_s > r1.admitted_s
    assert r1.time_to_steady_s == pytest.approx(r1.finished_s - 5.0)
    assert r0.time_to_steady_s == pytest.approx(r0.finished_s)
    assert rep["p50_time_to_steady_s"] == pytest.approx(percentile([r0.time_to_steady_s, r1.time_to_steady_s], 50))


def test_percentile_interpolates_between_ranks():
    assert percentile([3.0, 1.0, 2.0, 4.0], 50) == pytest.approx(2.5)
    assert percentile(list(range(101)), 99) == pytest.approx(99.0)
    assert percentile([7.0], 99) == 7.0


def test_finished_lattices_are_closed_and_populations_kept():
    jobs = [Job(i, 0.0, Script(8, 8, 8, [1e-3, 1e-9])) for i in range(3)]
    lats = []

    def lattice_factory(wl, p, s):
        lats.append(FakeLattice(wl))
        return lats[-1]

    srv = Server("f32", capacity=2, budget_bytes=1e12, keep_populations=True,
                 batch_factory=lambda c, p: FakeBatch(c, p), lattice_factory=lattice_factory)
    results, _ = srv.serve(jobs, closed_loop=True, clock=Clock())
    assert all(lat.closed for lat in lats)
    assert all(r.populations == ("state", 2) for r in results)
    assert [r.history for r in results] == [[1e-3, 1e-9]] * 3
