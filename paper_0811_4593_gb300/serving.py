"""Continuous-batching serving loop for lattice solves.

Jobs (lattice solves of different sizes, boundary velocities and relaxation times)
arrive over time. The server admits the job at the head of the queue as soon as a batch
slot is free and its device footprint fits the memory budget, keeps its populations
resident, and advances all admitted lattices together: one round is ``round_steps``
time steps of every resident lattice (a single CUDA-graph replay of persistent
launches, lbm_batch_step), ending in each lattice's residual and mass. After every
round the server retires the lattices that converged (residual below ``target``),
stopped improving (no new best residual for ``plateau_checks`` rounds), hit the step
cap, or diverged, and admits waiting jobs into the freed slots. Time to steady state is
measured from a job's arrival to the end of the round that retires it.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

from ._binding import Batch, Lattice

STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2}
COMPUTE_BYTES = {"f64": 8, "f32": 4, "f16": 4}


def footprint_bytes(nx: int, ny: int, nz: int, precision: str, scheme: str = "ab") -> int:
    """Device bytes one resident lattice holds: its population buffers (two for the A/B
    scheme, one for AA), the residual snapshot and partial sums, the face tables and the
    reduction scalars."""
    n = nx * ny * nz
    blocks = (n + 255) // 256
    faces = 2 * (ny * nz + nx * nz + nx * ny) * 48
    buffers = 1 if scheme == "aa" else 2
    return buffers * 19 * STORAGE_BYTES[precision] * n + 3 * COMPUTE_BYTES[precision] * n + 32 * blocks + faces + 32


@dataclass
class Job:
    """One solve: an id, its arrival time (seconds after the start) and the lattice
    (anything with nx, ny, nz, tau, rho0, kinds and utabs, as Lattice.from_workload
    takes)."""
    jid: int
    arrival_s: float
    workload: object


@dataclass
class JobResult:
    jid: int
    cells: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    steps: int
    residual: float
    mass: float
    status: str  # converged | plateau | step_cap | diverged
    history: list = field(default_factory=list)
    populations: object = None

    @property
    def time_to_steady_s(self) -> float:
        return self.finished_s - self.arrival_s


@dataclass
class _Active:
    job: Job
    lattice: Lattice
    admitted_s: float
    bytes: int
    steps: int = 0
    best: float = math.inf
    since_best: int = 0
    history: list = field(default_factory=list)


def percentile(values, q):
    if not values:
        return float("nan")
    v = sorted(values)
    k = (len(v) - 1) * q / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


class Server:
    def __init__(self, precision: str = "f32", capacity: int = 256, budget_bytes: float = 150e9,
                 round_steps: int = 100, max_steps: int = 20000, target: float = 1e-8, plateau_checks: int = 10,
                 plateau_ceiling: float = 1e-5, keep_populations: bool = False, scheme: str = "ab",
                 batch_factory=None, lattice_factory=None):
        """``batch_factory(capacity, precision)`` and ``lattice_factory(workload, precision,
        scheme)`` default to the library's Batch and Lattice.from_workload; other objects
        with the same methods can stand in for them (the scheduling logic is tested on the
        host that way)."""
        self.precision = precision
        self.capacity = int(capacity)
        self.budget = float(budget_bytes)
        self.round_steps = int(round_steps)
        self.max_steps = int(max_steps)
        self.target = float(target)
        self.plateau = int(plateau_checks)
        self.plateau_ceiling = float(plateau_ceiling)
        self.keep_populations = keep_populations
        self.scheme = scheme
        self.batch_factory = batch_factory or (lambda capacity, precision: Batch(capacity, precision))
        self.lattice_factory = lattice_factory or (
            lambda workload, precision, scheme: Lattice.from_workload(workload, precision, scheme=scheme))

    def serve(self, jobs, closed_loop: bool = False, clock=time.perf_counter, idle_sleep=0.001):
        """Run every job to completion. ``closed_loop`` ignores arrival times (all jobs
        queue at the start). Returns (results, report)."""
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival_s))
        waiting = collections.deque()
        active: dict[int, _Active] = {}
        results = []
        used = 0
        rounds = 0
        node_updates = 0
        peak_active = 0
        peak_bytes = 0
        batch = self.batch_factory(self.capacity, self.precision)
        t0 = clock()
        try:
            while pending or waiting or active:
                now = clock() - t0
                while pending and (closed_loop or pending[0].arrival_s <= now):
                    waiting.append(pending.popleft())
                # admission: FIFO, by free slot and memory footprint
                free = batch.free_slots()
                while waiting and free:
                    wl = waiting[0].workload
                    need = footprint_bytes(wl.nx, wl.ny, wl.nz, self.precision, self.scheme)
                    if need > self.budget:
                        raise ValueError(f"job {waiting[0].jid} needs {need} bytes, more than the whole budget")
                    if used + need > self.budget:
                        break
                    job = waiting.popleft()
                    lat = self.lattice_factory(job.workload, self.precision, self.scheme)
                    slot = free.pop(0)
                    batch.attach(slot, lat)
                    active[slot] = _Active(job, lat, clock() - t0, need)
                    used += need
                peak_active = max(peak_active, len(active))
                peak_bytes = max(peak_bytes, used)
                if not active:
                    if pending and not closed_loop:
                        time.sleep(max(0.0, min(idle_sleep, pending[0].arrival_s - (clock() - t0))))
                    continue
                batch.step(self.round_steps, residual=True)
                res = batch.results()
                rounds += 1
                end = clock() - t0
                for slot in list(active):
                    a = active[slot]
                    r, m, st = res[slot]
                    a.steps += self.round_steps
                    node_updates += a.lattice.cells * self.round_steps
                    a.history.append(r)
                    status = None
                    if st == -4:
                        status = "diverged"
                    elif r < self.target:
                        status = "converged"
                    else:
                        if r < a.best:
                            a.best, a.since_best = r, 0
                        else:
                            a.since_best += 1
                        if a.best < self.plateau_ceiling and a.since_best >= self.plateau:
                            status = "plateau"
                        elif a.steps >= self.max_steps:
                            status = "step_cap"
                    if status is None:
                        continue
                    batch.detach(slot)
                    pops = a.lattice.get_populations() if self.keep_populations else None
                    a.lattice.close()
                    used -= a.bytes
                    del active[slot]
                    results.append(JobResult(a.job.jid, a.lattice.cells, a.job.arrival_s, a.admitted_s, end, a.steps,
                                             r, m, status, a.history, pops))
        finally:
            for a in active.values():
                a.lattice.close()
            batch.close()
        wall = clock() - t0
        tts = [r.time_to_steady_s for r in results]
        ok = [r for r in results if r.status != "diverged"]
        by_status = collections.defaultdict(list)
        for r in results:
            by_status[r.status].append(r.time_to_steady_s)
        report = {
            "jobs": len(results),
            "wall_s": wall,
            "rounds": rounds,
            "node_updates": node_updates,
            "aggregate_mlups": node_updates / wall / 1e6 if wall > 0 else float("nan"),
            "jobs_per_s": len(results) / wall if wall > 0 else float("nan"),
            "p50_time_to_steady_s": percentile(tts, 50),
            "p99_time_to_steady_s": percentile(tts, 99),
            "status_counts": dict(collections.Counter(r.status for r in results)),
            "p50_time_by_status_s": {k: percentile(v, 50) for k, v in by_status.items()},
            "p99_time_by_status_s": {k: percentile(v, 99) for k, v in by_status.items()},
            "steps_p50": percentile([r.steps for r in results], 50),
            "steps_p99": percentile([r.steps for r in results], 99),
            "final_residual_p50": percentile([r.residual for r in ok], 50),
            "final_residual_p90": percentile([r.residual for r in ok], 90),
            "peak_active": peak_active,
            "peak_bytes": peak_bytes,
        }
        return sorted(results, key=lambda r: r.jid), report
