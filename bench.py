#!/usr/bin/env python3
"""Throughput benchmark of the fused D3Q19 sweep (MLUPS and HBM-roofline fraction).

Default workload: the 512^3 channel -- tau 0.8, uniform non-normal inflow and outflow
u = (0.04, 0.01, 0) at x = 0 and x = 511, periodic in y, no-slip walls at z = 0 and
z = 511 -- with FP32 population storage; 1000 timed steps after 200 warm-up steps and a
fused residual/mass reduction every 100 steps, as a steady-state solve runs. One time
step is one pass of the hot path over all 512^3 nodes. The populations (10.2 GB read
and 10.2 GB written per step) are far larger than the 129 MB L2, so no flush is needed.

Arms:
  --impl native     the CUDA library through its Python binding (default);
  --impl reference  the FP64 CPU oracle on the host cores, on a bounded sample of the
                    same workload (the paper publishes no implementation to run).
Under torchrun every rank runs an independent replica on its own GPU (the solve has
no data-path exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbm_inputs as inp  # noqa: E402

METRIC = "MLUPS & % HBM roofline (FP16/FP32 vs FP64) at stated error; serving p50/p99"
BYTES_PER_UPDATE = {"f64": 304, "f32": 152, "f16": 76}  # 19 loads + 19 stores per node update
FALLBACK_HBM_GBS = 6800.0


def workload(name: str):
    if name == "channel512":
        return inp.channel(512, 512, 512, 0.8, (0.04, 0.01, 0.0))
    if name == "channel256":  # the same channel at 256^3, for profiler captures
        return inp.channel(256, 256, 256, 0.8, (0.04, 0.01, 0.0))
    if name == "channel512x64":  # 512-node rows as at 512^3, 64 planes: profiler captures
        return inp.channel(512, 512, 64, 0.8, (0.04, 0.01, 0.0))
    if name == "duct":
        return inp.duct(256, 64, 64, 0.6, 0.05, 30.0)
    if name == "couette":
        return inp.couette()
    raise SystemExit(f"unknown workload {name}")


def describe(wl) -> str:
    if wl.name == "channel":
        return (f"channel {wl.nx}x{wl.ny}x{wl.nz}, tau {wl.tau}, uniform inflow/outflow u={wl.meta['u']} at x faces, "
                f"periodic y, no-slip z walls")
    if wl.name == "duct":
        return (f"square duct {wl.nx}x{wl.ny}x{wl.nz}, tau {wl.tau}, parabolic inlet/outlet peak {wl.meta['peak']} "
                f"tilted {wl.meta['angle_deg']} deg, no-slip y and z walls")
    return f"{wl.name} {wl.nx}x{wl.ny}x{wl.nz}, tau {wl.tau}"


def cpu_sample(wl):
    """The bounded oracle sample of a workload: same faces, tau and inflow, fewer planes."""
    if wl.name == "channel":
        s = inp.channel(128, 128, 16, wl.tau, wl.meta["u"])
        return s, f"channel {s.nx}x{s.ny}x{s.nz} (same faces, tau and inflow as the workload)"
    if wl.name == "duct":
        s = inp.duct(wl.nx, wl.ny, wl.nz, wl.tau, wl.meta["peak"], wl.meta["angle_deg"])
        return s, "the full duct"
    return wl, "the full lattice"


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return FALLBACK_HBM_GBS, "fallback"


def code_only(text: str) -> str:
    """C/C++/CUDA source with its comments, blank lines and the blanks around each line
    removed, so that the hash of the sweep source changes with the code and not with
    its comments or indentation. String and character literals are kept as they are."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = [ln.strip() for ln in "".join(out).splitlines()]
    return "\n".join(ln for ln in lines if ln)


def sweep_source_hash() -> str:
    """Hash of the sweep's code (kernels.cuh, d3q19.cuh; comments excluded): a profiled
    traffic figure is reported only while this matches the hash it was captured on."""
    h = hashlib.sha256()
    for f in ("kernels.cuh", "d3q19.cuh"):
        with open(os.path.join(ROOT, "paper_0811_4593_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, precision: str, wl_name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current sweep source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)[f"{kernel}/{precision}/{wl_name}"]
    except Exception:  # noqa: BLE001
        return None
    return rec["dram_bytes_per_launch"] if rec.get("source_sha") == sweep_source_hash() else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------
# native arm
# ------------------------------------------------------------------------------------

def timed_steps(lat, steps: int, resid_every: int, events: bool):
    """Issue `steps` time steps, a fused residual every `resid_every`. Returns CUDA
    events (on the lattice's stream) around each launch group -- one step, or one pair
    of steps for an AA lattice -- the group sizes, and the indices of residual groups."""
    import torch
    g = 2 if getattr(lat, "scheme", "ab") == "aa" else 1
    ngroups = steps // g
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(ngroups + 1)] if events else None
    if evs:
        evs[0].record(lat.stream)
    resid = []
    for i in range(ngroups):
        done = (i + 1) * g
        if resid_every and done % resid_every == 0:
            lat.step_residual(g)
            resid.append(i)
        else:
            lat.step(g)
        if evs:
            evs[i + 1].record(lat.stream)
    return evs, resid, g


def measure(lat, steps, warmup, resid_every, dist_ctx, clock_gpu=None):
    import torch
    timed_steps(lat, warmup, resid_every, events=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(clock_gpu).start() if clock_gpu is not None else None
    dist_ctx.barrier()
    torch.cuda.synchronize()
    l0 = lat.info()["kernel_launches"]
    evs, resid, g = timed_steps(lat, steps, resid_every, events=True)
    torch.cuda.synchronize()
    dist_ctx.barrier()
    clock = clocks.stop() if clocks else None
    launches = lat.info()["kernel_launches"] - l0
    n = len(evs) - 1
    total_ms = evs[0].elapsed_time(evs[n])
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(n)]
    after_sync = {i + 1 for i in resid}
    plain = [per[i] for i in range(n) if i not in resid and i not in after_sync]
    step_ms = (sum(plain) / len(plain) if plain else total_ms / n) / g
    return total_ms, step_ms, launches, clock


class Dist:
    """Rank bookkeeping for replicas: one process per GPU (NCCL), or gloo on CPU-only
    hosts. The only collectives are the barriers around the timed region and the
    max-over-ranks of the measured times; the solve itself exchanges nothing."""

    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = False
        self.backend = None

    def init(self, backend=None):
        import torch
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(self.local)
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": torch.device("cuda", self.local)} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)
            self.pg = True
        self.backend = backend

    def barrier(self):
        if self.pg:
            import torch.distributed as dist
            dist.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device="cuda" if self.backend == "nccl" else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            import torch.distributed as dist
            dist.destroy_process_group()


def whole_job_mlups(world: int, nodes: int, steps: int, max_ms: float) -> float:
    """Node updates of all replicas divided by the slowest replica's time."""
    return world * nodes * steps / (max_ms * 1e-3) / 1e6


# GB300's FP64 pipe: NVIDIA's 1.25 TFLOP/s FP64 figure is 2 DFMA per SM per clock at
# 152 SMs and 2.07 GHz, i.e. 2 FP64 instructions per SM per clock.
FP64_INST_PER_SM_CLOCK = 2.0


def profiled_fp64_per_node(wl_name: str):
    """FP64 instructions per node update of the FP64 sweep from the committed ncu
    counters, if they were taken on the current sweep source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)[f"sweep/f64/{wl_name}"]
    except Exception:  # noqa: BLE001
        return None
    return rec.get("fp64_inst_per_node") if rec.get("source_sha") == sweep_source_hash() else None


def sweep_kernel_name(wl, precision, scheme="ab"):
    """The kernel that runs the plain (non-residual) steps of a lattice."""
    if precision == "f16" and wl.nx % 2 == 0 and getattr(wl, "solid", None) is None \
            and getattr(wl, "force", None) is None:
        if wl.nx % 8 == 0 and wl.nx >= 256:
            return "sweep_rows_kernel<f16>" + ("" if scheme == "ab" else " (AA steps)")
        return "sweep_pair_kernel<f16>" + ("" if scheme == "ab" else " (AA steps)")
    return f"sweep_kernel<{precision}>"


def run_variant(wl, precision, steps, warmup, resid_every, dist_ctx, clocks=None, scheme="ab"):
    import torch

    import paper_0811_4593_gb300 as lbm
    with lbm.Lattice.from_workload(wl, precision, scheme=scheme) as lat:
        total_ms, step_ms, launches, _ = measure(lat, steps, warmup, resid_every, dist_ctx)
    hbm, _ = measured_hbm_peak()
    ach = BYTES_PER_UPDATE[precision] * wl.cells / (step_ms * 1e-3) / 1e9
    out = {"mlups": wl.cells * steps / (total_ms * 1e-3) / 1e6, "ms_per_step": total_ms / steps,
           "sweep_ms": step_ms, "achieved_gbs": ach, "frac": ach / hbm, "steps": steps,
           "bytes_per_update": BYTES_PER_UPDATE[precision], "scheme": scheme,
           "kernel": sweep_kernel_name(wl, precision, scheme),
           "resident_bytes_per_node": BYTES_PER_UPDATE[precision] // (2 if scheme == "aa" else 1)}
    if precision == "f64":
        # the FP64 sweep is bound by the FP64 pipe, not by HBM: its peak is the measured
        # FP64 FMA rate of this device (thread-level operations per second; FP64 adds and
        # multiplies issue at the same rate), the spec-derived figure is context only
        from paper_0811_4593_gb300._binding import fp64_fma_rate
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        nominal = FP64_INST_PER_SM_CLOCK * sms * mhz * 1e6 / 1e9
        clk = ClockSampler(torch.cuda.current_device()).start()
        rate, probe_ms = fp64_fma_rate(12000)
        probe_clock = clk.stop()
        peak = rate / 1e9
        per_node = profiled_fp64_per_node("channel256")
        alu = {"bound": "alu", "unit": "G FP64 inst/s", "peak": round(peak, 1), "peak_source": "measured",
               "peak_basis": (f"lbm_fp64_fma_rate: 8 independent DFMA chains per thread on every resident warp, "
                              f"{probe_ms:.1f} ms, SM clock {probe_clock.get('sm_mhz')} MHz"),
               "nominal": round(nominal, 1),
               "nominal_basis": f"{FP64_INST_PER_SM_CLOCK:g} FP64 inst / SM / clock x {sms} SMs x {mhz:g} MHz",
               "fp64_inst_per_node": per_node}
        if per_node:
            a = per_node * wl.cells / (step_ms * 1e-3) / 1e9
            alu.update(achieved=round(a, 1), frac=round(a / peak, 4))
        out["roofline"] = alu
    return out


def e2e_run(wl, precision, steps, resid_every, dist_ctx, scheme="ab"):
    """Same solve through the public API with host buffers: upload the initial
    populations from pinned host memory, run the steps, read the density and velocity
    fields back to pinned host memory -- all inside the timed region."""
    import torch

    import paper_0811_4593_gb300 as lbm
    with lbm.Lattice.from_workload(wl, precision, scheme=scheme) as lat:
        dt = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16}[precision]
        mdt = torch.float64 if precision == "f64" else torch.float32
        f_host = torch.empty((19, wl.nz, wl.ny, wl.nx), dtype=dt, pin_memory=True)
        lat.get_populations(out=f_host)          # the initial state, staged on the host
        rho_dev = torch.empty((wl.nz, wl.ny, wl.nx), dtype=mdt, device="cuda")
        u_dev = torch.empty((3, wl.nz, wl.ny, wl.nx), dtype=mdt, device="cuda")
        rho_host = torch.empty(rho_dev.shape, dtype=mdt, pin_memory=True)
        u_host = torch.empty(u_dev.shape, dtype=mdt, pin_memory=True)
        torch.cuda.synchronize()
        dist_ctx.barrier()
        t0 = time.perf_counter()
        lat.set_populations(f_host)
        timed_steps(lat, steps, resid_every, events=False)
        lat.macros(rho_dev, u_dev)
        rho_host.copy_(rho_dev, non_blocking=True)
        u_host.copy_(u_dev, non_blocking=True)
        torch.cuda.synchronize()
        dt_s = time.perf_counter() - t0
        dist_ctx.barrier()
        h2d = f_host.numel() * f_host.element_size()
        d2h = rho_host.numel() * rho_host.element_size() + u_host.numel() * u_host.element_size() + \
            32 * (steps // resid_every if resid_every else 0)
    return dt_s, h2d, d2h


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), with the architecture."""
    import platform
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001 - lscpu missing
        pass
    if not name:
        try:
            fields = {}
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if ":" in line:
                        k, v = line.split(":", 1)
                        fields.setdefault(k.strip().lower(), v.strip())
            name = fields.get("model name") or (
                f"implementer {fields['cpu implementer']} part {fields['cpu part']}" if "cpu part" in fields else None)
        except OSError:
            pass
    return f"{name or 'unknown'} ({platform.machine()})"


def cpu_baseline(wl, seconds: float):
    import oracle
    sample, text = cpu_sample(wl)
    olat = oracle.Lattice.from_workload(sample)
    f = oracle.init_equilibrium(olat, sample.rho0)
    t0 = time.perf_counter()
    n = 0
    while True:
        f = oracle.step(olat, f)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": sample.cells * n / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
            "cpu": cpu_model(), "sample": f"{text}, {n} FP64 steps from rest in {dt:.1f} s"}


def native(args):
    import torch

    import paper_0811_4593_gb300 as lbm
    from paper_0811_4593_gb300 import build as lib_build
    if args.sweep_scheme == "aa" and (args.steps % 2 or args.warmup % 2 or args.resid_every % 2):
        raise SystemExit("an AA lattice advances in pairs of steps: give even --steps, --warmup and --resid-every")
    d = Dist()
    if d.rank == 0 or not os.path.exists(lib_build.LIB):
        lib_build.build()
    d.init("nccl")
    wl = workload(args.workload)
    hbm, hbm_src = measured_hbm_peak()
    with lbm.Lattice.from_workload(wl, args.precision, scheme=args.sweep_scheme) as lat:
        total_ms, sweep_ms, launches, clock = measure(lat, args.steps, args.warmup, args.resid_every, d,
                                                      clock_gpu=d.local)
    total_ms = d.max(total_ms)
    sweep_ms = d.max(sweep_ms)
    value = whole_job_mlups(d.world, wl.cells, args.steps, total_ms)
    achieved = BYTES_PER_UPDATE[args.precision] * wl.cells / (sweep_ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": d.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": describe(wl), "nodes": wl.cells, "precision": f"{args.precision} population storage",
                   "streaming": "A/B (two arrays)" if args.sweep_scheme == "ab" else "AA (one array)",
                   "residual_every": args.resid_every, "parallelism": "replicas" if d.world > 1 else "single GPU",
                   "l2": f"inputs larger than L2: {BYTES_PER_UPDATE[args.precision] * wl.cells / 2e9:.1f} GB of "
                         f"populations read per step (no flush needed)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "peak_source": hbm_src,
                     "traffic": profiled_traffic("sweep", args.precision, args.workload)
                     if args.sweep_scheme == "ab" else None,
                     "kernel": sweep_kernel_name(wl, args.precision, args.sweep_scheme),
                     "bytes_per_update": BYTES_PER_UPDATE[args.precision], "updates_per_launch": wl.cells,
                     "sweep_ms": round(sweep_ms, 4)},
        "gpu_launches": launches,
        "clocks": clock,
    }
    if not args.no_e2e:
        dt_s, h2d, d2h = e2e_run(wl, args.precision, args.steps, args.resid_every, d, args.sweep_scheme)
        dt_s = d.max(dt_s)
        out["e2e"] = {"value": round(whole_job_mlups(d.world, wl.cells, args.steps, dt_s * 1e3), 1), "unit": "MLUPS",
                      "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}
    if d.world == 1 and not args.no_variants and args.workload == "channel512":
        torch.cuda.empty_cache()
        vs = {}
        for p in ("f16", "f64"):
            if p != args.precision:
                vs[p] = run_variant(wl, p, args.variant_steps, 20, args.resid_every, d, clock)
                torch.cuda.empty_cache()
        for p in dict.fromkeys((args.precision, "f16")):
            vs[f"{p}_aa"] = run_variant(wl, p, args.variant_steps, 20, args.resid_every, d, clock, scheme="aa")
            torch.cuda.empty_cache()
        out["variants"] = vs
    if d.world == 1 and args.serving_requests > 0:
        torch.cuda.empty_cache()
        rec = serving_run(args.precision, args.serving_requests, args.serving_capacity_requests, args.slots,
                          args.budget_gb, args.resid_every, args.max_steps, args.target, args.scheme,
                          clock_gpu=d.local)
        rec["batched_sweep"] = batched_sweep_roofline(args.precision)
        rec["note"] = ("bounded serving leg of the default run; bench.py --serving runs the 2000-request mix")
        out["serving"] = rec
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    d.close()
    if d.rank == 0:
        print(json.dumps(out), flush=True)


def batched_sweep_roofline(precision: str, nlat: int = 40, steps: int = 100, warmup: int = 20):
    """The batched sweep on a fixed serving mix: the first `nlat` requests of the seed-1
    stream resident together, `steps` batched A/B steps timed with CUDA events on the
    batch's stream. Bytes are the algorithmic 19 loads + 19 stores per node update."""
    import torch

    import paper_0811_4593_gb300 as lbm
    reqs = inp.serving_requests(nlat, 1, 1.0)
    stream = torch.cuda.Stream()
    lats = []
    with lbm.Batch(nlat, precision, stream=stream) as b:
        try:
            for i, r in enumerate(reqs):
                lats.append(lbm.Lattice.from_workload(inp.request_workload(r), precision))
                b.attach(i, lats[-1])
            grid = b.info()["grid"]
            b.step(warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
        finally:
            for lat in lats:
                lat.close()
    nodes = sum(r.cells for r in reqs)
    hbm, src = measured_hbm_peak()
    ach = BYTES_PER_UPDATE[precision] * nodes / (ms * 1e-3) / 1e9
    return {"kernel": f"sweep_batched_kernel<{precision}>", "lattices": nlat, "updates_per_launch": nodes,
            "grid": grid, "launch_ms": round(ms, 4), "mlups": round(nodes / (ms * 1e-3) / 1e6, 1), "bound": "hbm",
            "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
            "peak_source": src, "bytes_per_update": BYTES_PER_UPDATE[precision],
            "traffic": profiled_traffic("batched", precision, f"serving{nlat}"),
            "mix": f"first {nlat} requests of the seed-1 serving stream, all resident"}


def serving_run(precision: str, requests: int, capacity_requests: int, slots: int, budget_gb: float,
                round_steps: int, max_steps: int, target: float, scheme: str, clock_gpu=None) -> dict:
    """The serving mix: capacity (jobs/s) from a closed-loop run of `capacity_requests`
    of the seed-1 request stream, then `requests` of the seed-0 stream with Poisson
    arrivals at 70 % of that capacity. Returns the serving record (p50/p99 time to
    steady state, aggregate MLUPS, how the jobs ended, clocks during the run)."""
    import torch

    from paper_0811_4593_gb300.serving import Job, Server
    kw = dict(capacity=slots, budget_bytes=budget_gb * 1e9, round_steps=round_steps,
              max_steps=max_steps, target=target, plateau_checks=10, scheme=scheme)
    clocks = ClockSampler(clock_gpu).start() if clock_gpu is not None else None
    cap_reqs = inp.serving_requests(capacity_requests, 1, 1.0)
    cap_jobs = [Job(r.rid, 0.0, inp.request_workload(r)) for r in cap_reqs]
    _, cap = Server(precision, **kw).serve(cap_jobs, closed_loop=True)
    capacity = cap["jobs_per_s"]
    rate = 0.7 * capacity
    reqs = inp.serving_requests(requests, 0, rate)
    jobs = [Job(r.rid, r.arrival_s, inp.request_workload(r)) for r in reqs]
    torch.cuda.synchronize()
    _, rep = Server(precision, **kw).serve(jobs)
    clock = clocks.stop() if clocks else None
    return {"requests": requests, "p50_time_to_steady_s": round(rep["p50_time_to_steady_s"], 3),
            "p99_time_to_steady_s": round(rep["p99_time_to_steady_s"], 3),
            "aggregate_mlups": round(rep["aggregate_mlups"], 1),
            "jobs": rep["jobs"], "wall_s": round(rep["wall_s"], 2),
            "capacity_jobs_per_s": round(capacity, 3), "arrival_rate_per_s": round(rate, 3),
            "capacity_run": {"requests": capacity_requests, "jobs": cap["jobs"], "wall_s": round(cap["wall_s"], 2),
                             "aggregate_mlups": round(cap["aggregate_mlups"], 1),
                             "status_counts": cap["status_counts"]},
            "status_counts": rep["status_counts"],
            "p50_time_by_status_s": {k: round(v, 3) for k, v in rep["p50_time_by_status_s"].items()},
            "p99_time_by_status_s": {k: round(v, 3) for k, v in rep["p99_time_by_status_s"].items()},
            "steady_state_rule": (f"retired at residual < {target} (converged), no new best over 10 checks once "
                                  f"below 1e-5 (plateau), {max_steps} steps (step_cap) or a bad node (diverged)"),
            "peak_active": rep["peak_active"], "peak_gb": round(rep["peak_bytes"] / 1e9, 2),
            "steps_p50": rep["steps_p50"], "steps_p99": rep["steps_p99"],
            "final_residual_p50": rep["final_residual_p50"], "final_residual_p90": rep["final_residual_p90"],
            "slots": slots, "budget_gb": budget_gb, "round_steps": round_steps, "scheme": scheme,
            "precision": precision, "clocks": clock}


def serving(args):
    """The full serving mix as its own JSON line (2000 requests by default)."""
    import torch

    from paper_0811_4593_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rec = serving_run(args.precision, args.requests, args.capacity_requests, args.slots, args.budget_gb,
                      args.resid_every, args.max_steps, args.target, args.scheme,
                      clock_gpu=int(os.environ.get("LOCAL_RANK", "0")))
    rec["batched_sweep"] = batched_sweep_roofline(args.precision)
    out = {"metric": METRIC, "value": rec["aggregate_mlups"], "unit": "MLUPS", "n_gpus": 1,
           "higher_is_better": True, "dtype": args.precision, "data": "synthetic", "mode": "serving",
           "config": {"workload": f"serving mix: {args.requests} duct/channel requests, dims log-uniform 32..192, "
                                  f"speed U(0.01,0.08), angle U(0,45 deg), tau U(0.55,1.5), Poisson arrivals at "
                                  f"0.7 x capacity, residual target {args.target} or {args.max_steps} steps",
                      "slots": args.slots, "budget_gb": args.budget_gb, "round_steps": args.resid_every},
           "serving": rec}
    print(json.dumps(out), flush=True)


def tilted_poiseuille(wl):
    """eq. pois: v0 [1 - ((x - x0 - g (z - z0)) / dx)^2] along the channel axis, on the
    fluid nodes of a tilted-channel workload (zero on solid nodes)."""
    import numpy as np
    m = wl.meta
    x = np.arange(wl.nx)[None, None, :]
    z = np.arange(wl.nz)[:, None, None]
    d = (x - m["x0"] - m["gamma"] * (z - m["z0"])) / m["half_width"] + np.zeros((1, wl.ny, 1))
    prof = np.where(wl.solid == 0, m["u0"] * (1 - d * d), 0.0)
    return prof[None] * np.array(m["direction"])[:, None, None, None]


def tilted_xi(wl, u, near_planes: bool = False):
    """eq. deferr as the mean of |v - v^P| / |v^P| over fluid nodes: all of them, or
    (near_planes) those within one channel width (20 nodes, times the scale) of the
    inflow and outflow planes -- the two readings of the paper's averaging volume."""
    import numpy as np
    vp = tilted_poiseuille(wl)
    sel = wl.solid == 0
    if near_planes:
        z = np.arange(wl.nz)[:, None, None] + np.zeros((1, wl.ny, wl.nx))
        w = 20 * wl.meta["scale"]
        sel = sel & ((z < w) | (z >= wl.nz - w))
    num = np.sqrt(((u - vp) ** 2).sum(0))[sel]
    den = np.sqrt((vp ** 2).sum(0))[sel]
    return float((num / den).mean())


def study_tilted(args):
    """The paper's tilted-channel comparison: xi of the on-site closure (GPU, FP64) at
    the paper's size and at twice its resolution, of the straight channel, of the inflow
    restricted to the plane normal, and of the N = 0 closure (FP64 oracle on the host:
    a comparison closure the CUDA path does not carry). The normal-only inflow is taken
    both as the z component of the profile and as its full speed along z."""
    import torch

    import paper_0811_4593_gb300 as lbm
    from paper_0811_4593_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cases = [("on_site", inp.tilted_channel(), 20000), ("on_site_2x", inp.tilted_channel(scale=2), 80000),
             ("straight", inp.tilted_channel(shift=0), 20000),
             ("normal_only", inp.tilted_channel(normal_only=True), 20000),
             ("normal_only_magnitude", inp.tilted_channel(normal_only="magnitude"), 20000)]
    out = {"study": "tilted channel (Sec. Numerical Results)", "tau": 1.0, "u0": 0.01,
           "xi": {}, "xi_near_planes": {}, "seconds": {}}
    for name, wl, steps in cases:
        t0 = time.perf_counter()
        with lbm.Lattice.from_workload(wl, "f64") as lat:
            lat.step(steps)
            _, u = lat.macros()
            u = u.cpu().numpy()
        out["xi"][name] = round(tilted_xi(wl, u), 5)
        out["xi_near_planes"][name] = round(tilted_xi(wl, u, near_planes=True), 5)
        out["seconds"][name] = round(time.perf_counter() - t0, 2)
    if not args.no_cpu_baseline:
        import oracle
        wl = inp.tilted_channel()
        t0 = time.perf_counter()
        olat = oracle.Lattice.from_workload(wl)
        f = oracle.run(olat, oracle.init_equilibrium(olat), 20000, form=oracle.FORM_COMPACT_NO_N)
        _, u = oracle.macros(olat, f)
        out["xi"]["n_zero_oracle"] = round(tilted_xi(wl, u), 5)
        out["xi_near_planes"]["n_zero_oracle"] = round(tilted_xi(wl, u, near_planes=True), 5)
        out["seconds"]["n_zero_oracle"] = round(time.perf_counter() - t0, 1)
    out["paper"] = {"on_site": 0.0996, "n_zero": 0.126, "normal_only": 0.175, "on_site_2x": 0.051, "straight": 0.00235}
    print(json.dumps(out), flush=True)


def study_duct(args):
    """The paper's square-channel study: pressure planes at both ends of an n x n duct
    with no-slip walls, edges and corners; relative L2 error of the mid-duct velocity
    against eq. squarechannel (50 terms, local pressure gradient, eta from eq. visc)
    for widths 8 .. 64 (FP64, on the GPU)."""
    import numpy as np
    import torch

    import paper_0811_4593_gb300 as lbm
    from paper_0811_4593_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))

    def series(n, terms=50):
        b = n - 1.0
        s_ = np.arange(n) - (n - 1) / 2.0
        X, Y = np.meshgrid(s_, s_, indexing="ij")
        C = np.zeros_like(X)
        for m in range(terms):
            k = 2 * m + 1
            C += (-1) ** m * np.cosh(k * np.pi * X / b) * np.cos(k * np.pi * Y / b) / (k ** 3 * np.cosh(k * np.pi / 2))
        return b * b / 4 - Y ** 2 - C * 8 * b * b / np.pi ** 3

    rows = []
    for n in (9, 13, 17, 25, 33, 49, 65):
        length = 3 * n
        wl = inp.pressure_duct(n, length, 1.0, 1.002, 0.998)
        t0 = time.perf_counter()
        with lbm.Lattice.from_workload(wl, "f64") as lat:
            lat.step(14 * n * n)
            rho, u = lat.macros()
            rho, u = rho.cpu().numpy(), u.cpu().numpy()
        xm = length // 2
        grad = (rho[:, :, xm + 1].mean() - rho[:, :, xm - 1].mean()) / 2.0 / 3.0
        eta = rho[:, :, xm].mean() * 0.5 / 3.0
        an = -grad / (2 * eta) * series(n)
        err = float(np.sqrt(((u[0][:, :, xm] - an) ** 2).mean() / (an ** 2).mean()))
        rows.append({"width": n - 1, "nodes": wl.cells, "steps": 14 * n * n, "l2_rel_error": err,
                     "seconds": round(time.perf_counter() - t0, 2)})
    for i in range(1, len(rows)):
        rows[i]["slope"] = round(float(np.log(rows[i - 1]["l2_rel_error"] / rows[i]["l2_rel_error"]) /
                                       np.log(rows[i]["width"] / rows[i - 1]["width"])), 3)
    print(json.dumps({"study": "pressure-driven square duct (Sec. Numerical Results)", "tau": 1.0,
                      "rho_in_out": [1.002, 0.998], "rows": rows, "paper_slope": 2}), flush=True)


def _gpu_study_setup():
    import torch

    from paper_0811_4593_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))


def study_poiseuille(args):
    """Plane Poiseuille sweep (4 x 4 x Lz, Lz = 16 .. 256, tau 0.55 / 1 / 1.5, peak
    0.02): the prescribed parabola at inlet and outlet is an exact steady solution of
    the method. Per case: FP64 steps until the residual falls below 1e-10; the FP64
    oracle run for the same steps; FP32 and binary16 runs of the same length. Reported:
    L2 error against the parabola, maximum velocity difference to the oracle, the
    residual reached, or the step at which a run diverged."""
    import numpy as np

    import oracle
    import paper_0811_4593_gb300 as lbm
    _gpu_study_setup()
    rows = []
    for tau in (0.55, 1.0, 1.5):
        for lz in (16, 32, 64, 128, 256):
            wl = inp.poiseuille(lz, tau, 0.02)
            exact = 0.02 * inp.parabola(lz)[:, None, None] * np.ones((1, wl.ny, wl.nx))
            row = {"tau": tau, "lz": lz}
            steps = None
            for prec in ("f64", "f32", "f16"):
                if prec != "f64" and steps is None:
                    row[prec] = {"skipped": "the FP64 run diverged"}
                    continue
                t0 = time.perf_counter()
                res = None
                with lbm.Lattice.from_workload(wl, prec) as lat:
                    try:
                        done = 0
                        if prec == "f64":
                            while done < 400_000:
                                r, _ = lat.step_residual(100)
                                done += 100
                                if r < 1e-10:
                                    break
                            steps = done
                        else:
                            while done < steps:
                                r, _ = lat.step_residual(min(100, steps - done))
                                done += min(100, steps - done)
                        res = r
                        _, u = lat.macros()
                        u = u.double().cpu().numpy()
                    except lbm.LBMDiverged:
                        row[prec] = {"diverged_at_step": lat.info()["steps"]}
                        if prec == "f64":
                            steps = None
                        continue
                l2 = float(np.sqrt(((u[0] - exact) ** 2).sum() / (exact ** 2).sum()))
                row[prec] = {"l2_vs_parabola": l2, "residual": res, "steps": done,
                             "max_transverse": float(np.abs(u[1:]).max()), "seconds": round(time.perf_counter() - t0, 2)}
                if prec == "f64":
                    olat = oracle.Lattice.from_workload(wl)
                    f = oracle.run(olat, oracle.init_equilibrium(olat), steps)
                    _, uo = oracle.macros(olat, f)
                    row["oracle_u"] = uo
                if "oracle_u" in row:
                    row[prec]["max_vs_oracle"] = float(np.abs(u - row["oracle_u"]).max() / 0.02)
            row.pop("oracle_u", None)
            rows.append(row)
    print(json.dumps({"study": "plane Poiseuille sweep (Sec. Numerical Results)", "rows": rows}), flush=True)


def study_duct_config(args):
    """The 256 x 64 x 64 duct (inlet and outlet product parabola, peak 0.05 at 30
    degrees, resting walls), 20000 steps at tau 0.6 and 1.0 in FP64 and FP32 on the GPU
    against the FP64 oracle run on the host cores; the mid-duct axial velocity against
    eq. squarechannel at matched flux."""
    import numpy as np

    import oracle
    import paper_0811_4593_gb300 as lbm
    _gpu_study_setup()

    def series(ny, nz, terms=50):
        b = ny - 1.0
        ys = np.arange(ny) - (ny - 1) / 2.0
        zs = np.arange(nz) - (nz - 1) / 2.0
        Z, Y = np.meshgrid(zs, ys, indexing="ij")
        C = np.zeros_like(Y)
        for m in range(terms):
            k = 2 * m + 1
            C += (-1) ** m * np.cosh(k * np.pi * Z / b) * np.cos(k * np.pi * Y / b) / (k ** 3 * np.cosh(k * np.pi / 2))
        return b * b / 4 - Y ** 2 - C * 8 * b * b / np.pi ** 3

    steps = int(getattr(args, "study_steps", 0) or 20000)
    out = {"study": f"duct 256x64x64, {steps} steps", "rows": []}
    for tau in (0.6, 1.0):
        wl = inp.duct(256, 64, 64, tau, 0.05, 30.0)
        t0 = time.perf_counter()
        olat = oracle.Lattice.from_workload(wl)
        ref = oracle.run(olat, oracle.init_equilibrium(olat), steps)
        _, uo = oracle.macros(olat, ref)
        row = {"tau": tau, "oracle_seconds": round(time.perf_counter() - t0, 1), "oracle_threads": oracle.threads()}
        scale = np.abs(uo).max()
        for prec in ("f64", "f32"):
            t0 = time.perf_counter()
            with lbm.Lattice.from_workload(wl, prec) as lat:
                lat.step(steps)
                _, u = lat.macros()
                u = u.double().cpu().numpy()
            row[prec] = {"max_vs_oracle": float(np.abs(u - uo).max() / scale),
                         "seconds": round(time.perf_counter() - t0, 2)}
        mid = uo[:, :, :, wl.nx // 2]                       # [3][z][y]
        axial = mid[0] * math.cos(math.radians(30)) + mid[1] * math.sin(math.radians(30))
        shape = series(wl.ny, wl.nz)
        an = shape * (axial.sum() / shape.sum())           # matched flux
        row["mid_duct_l2_vs_squarechannel"] = float(np.sqrt(((axial - an) ** 2).sum() / (an ** 2).sum()))
        out["rows"].append(row)
    print(json.dumps(out), flush=True)


def study_force(args):
    """The paper's body-force check: 32^3, walls on the x faces, periodic y and z, tau 2
    and 1: maximum deviation of the velocity after the boundary rule from eq. poiseuille
    (viscosity from eq. visc) and the velocity on the wall nodes, on the GPU in FP64 and
    FP32; the same with the transverse corrections set to zero (FP64 oracle)."""
    import numpy as np

    import oracle
    import paper_0811_4593_gb300 as lbm
    _gpu_study_setup()
    rows = []
    for tau, steps, force in ((2.0, 8000, 1e-6), (1.0, 22000, 1e-6), (2.0, 8000, 1e-5), (1.0, 22000, 1e-5)):
        wl = inp.force_poiseuille(n=32, tau=tau, force=force, wall_axis=0, flow_axis=2, other=None)
        F = wl.force[2]
        x = np.arange(wl.nx)
        h = (wl.nx - 1) / 2.0
        row = {"tau": tau, "steps": steps, "force": F}
        for prec in ("f64", "f32", "oracle_n_zero"):
            if prec == "oracle_n_zero":
                olat = oracle.Lattice.from_workload(wl)
                f = oracle.run(olat, oracle.init_equilibrium(olat), steps, form=oracle.FORM_COMPACT_NO_N)
                rho, u = oracle.macros(olat, f)
            else:
                with lbm.Lattice.from_workload(wl, prec) as lat:
                    lat.step(steps)
                    rho, u = lat.macros()
                    rho, u = rho.double().cpu().numpy(), u.double().cpu().numpy()
            u_pre = u[2] - F / rho
            exact = F / (2.0 * rho * (tau - 0.5) / 3.0) * (h * h - (x - h) ** 2)
            row[prec] = {"max_rel_error": float(np.abs(u_pre - exact).max() / exact.max()),
                         "wall_velocity": float(np.abs(u_pre[:, :, [0, -1]]).max()),
                         "u_max": float(exact.max())}
        rows.append(row)
    print(json.dumps({"study": "body-force Poiseuille 32^3 (eq. gravity, eq. poiseuille)", "rows": rows}),
          flush=True)


def study_batched(args):
    """The batched sweep alone on its fixed serving mix (the first 40 requests of the
    seed-1 stream, all resident): launch time, MLUPS and HBM-roofline fraction."""
    _gpu_study_setup()
    print(json.dumps({"study": "batched sweep on a serving mix", **batched_sweep_roofline(args.precision)}), flush=True)


def study_configs(args):
    """Throughput of the small configurations (Couette 8x8x17, 5000 steps; plane
    Poiseuille 4x4x256, tau 1, 15100 steps) on the GPU in each storage type and in the
    FP64 oracle on the host cores, with the GPU-vs-oracle velocity error."""
    import numpy as np
    import torch

    import oracle
    import paper_0811_4593_gb300 as lbm
    _gpu_study_setup()
    rows = []
    for name, wl, steps in (("couette 8x8x17", inp.couette(), 5000),
                            ("poiseuille 4x4x256 tau 1", inp.poiseuille(256, 1.0), 15100)):
        olat = oracle.Lattice.from_workload(wl)
        t0 = time.perf_counter()
        ref = oracle.run(olat, oracle.init_equilibrium(olat), steps)
        dt = time.perf_counter() - t0
        _, uo = oracle.macros(olat, ref)
        row = {"config": name, "steps": steps, "nodes": wl.cells,
               "oracle": {"mlups": wl.cells * steps / dt / 1e6, "threads": oracle.threads()}}
        for prec in ("f64", "f32", "f16"):
            with lbm.Lattice.from_workload(wl, prec) as lat:
                lat.step(10)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(lat.stream)
                lat.step(steps - 10)
                e1.record(lat.stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                _, u = lat.macros()
                u = u.double().cpu().numpy()
            row[prec] = {"mlups": wl.cells * (steps - 10) / (ms * 1e-3) / 1e6,
                         "max_vs_oracle": float(np.abs(u - uo).max() / np.abs(uo).max())}
        rows.append(row)
    print(json.dumps({"study": "small configurations", "rows": rows}), flush=True)


def reference(args):
    """The FP64 oracle on the host cores, `--steps` timed steps after `--warmup` on the
    bounded sample of the workload; rank 0 only."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    wl = workload(args.workload)
    sample, text = cpu_sample(wl)
    olat = oracle.Lattice.from_workload(sample)
    f = oracle.init_equilibrium(olat, sample.rho0)
    f = oracle.run(olat, f, args.warmup)
    t0 = time.perf_counter()
    f = oracle.run(olat, f, args.steps)
    dt = time.perf_counter() - t0
    value = sample.cells * args.steps / dt / 1e6
    out = {"metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": describe(wl), "nodes": wl.cells, "precision": "f64 (oracle)",
                      "parallelism": "host cores"},
           "cpu_baseline": {"value": round(value, 2), "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                            "cpu": cpu_model(),
                            "sample": f"{text}, {args.steps} FP64 steps after {args.warmup} warm-up steps"},
           "e2e": {"value": round(value, 2), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="channel512",
                    choices=["channel512", "channel256", "channel512x64", "duct", "couette"])
    ap.add_argument("--sweep-scheme", choices=["ab", "aa"], default="ab",
                    help="streaming scheme of the benchmarked lattice (AA: step pairs, so even step counts)")
    ap.add_argument("--precision", default="f32", choices=["f32", "f16", "f64"])
    ap.add_argument("--resid-every", type=int, default=100)
    ap.add_argument("--variant-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", action="store_true", help="run the serving mix instead of the sweep benchmark")
    ap.add_argument("--study", choices=["tilted", "duct", "poiseuille", "duct-config", "force", "configs", "batched"],
                    help="run a reproduction study instead of the benchmark")
    ap.add_argument("--study-steps", type=int, default=0, help="steps of the duct-config study (default 20000)")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--capacity-requests", type=int, default=200)
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="requests of the serving leg of the default run (0: no serving leg)")
    ap.add_argument("--serving-capacity-requests", type=int, default=100,
                    help="closed-loop requests that measure capacity in the serving leg of the default run")
    ap.add_argument("--slots", type=int, default=512)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--max-steps", type=int, default=20000)
    ap.add_argument("--target", type=float, default=1e-8)
    ap.add_argument("--scheme", choices=["ab", "aa"], default="ab", help="streaming scheme of the serving lattices")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference(args)
    elif args.study == "tilted":
        study_tilted(args)
    elif args.study == "duct":
        study_duct(args)
    elif args.study == "poiseuille":
        study_poiseuille(args)
    elif args.study == "duct-config":
        study_duct_config(args)
    elif args.study == "force":
        study_force(args)
    elif args.study == "configs":
        study_configs(args)
    elif args.study == "batched":
        study_batched(args)
    elif args.serving:
        serving(args)
    else:
        native(args)


if __name__ == "__main__":
    main()
