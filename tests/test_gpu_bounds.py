"""GPU run of the index-checking debug build (LBM_DEBUG_BOUNDS): a battery of lattices
through every sweep variant -- single-node, paired and row-staged, A/B and AA, residual steps,
velocity, pressure and periodic faces, solid nodes and on-site geometry codes, a body
force, a batch -- must meet no out-of-range population, face-table or geometry-word
index. The debug library runs in a child process (LBM_LIBRARY points at it)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

BATTERY = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import lbm_inputs as inp
import paper_0811_4593_gb300 as lbm
from paper_0811_4593_gb300._binding import debug_bounds_errors
torch.cuda.set_device(0)
ran = []
def run(wl, prec, scheme="ab", steps=6):
    with lbm.Lattice.from_workload(wl, prec, scheme=scheme) as lat:
        lat.step(steps)
        lat.step_residual(2)
        lat.macros()
    ran.append((wl.name, prec, scheme))
for prec in ("f16", "f32", "f64"):
    for scheme in ("ab", "aa"):
        run(inp.channel(32, 20, 21, 0.7, (0.04, 0.01, 0.0)), prec, scheme)        # even nx, walled x
        run(inp.duct(37, 19, 23, 0.8, 0.05, 30.0), prec, scheme)                 # odd nx
        run(inp.random_pressure_workload(28, 12, 10, 11, 0.9), prec, scheme)     # pressure faces
        run(inp.make_workload("periodic", 10, 7, 5, 0.6, [None] * 6), prec, scheme)
        run(inp.random_face_workload(29, 4, 3, 3, 1.0, (False, False, False)), prec, scheme)
        run(inp.duct(264, 9, 7, 0.8, 0.05, 30.0), prec, scheme)                   # binary16: row-staged
for prec in ("f16", "f32", "f64"):
    for axis in range(3):
        flow = [a for a in range(3) if a != axis][0]
        run(inp.pillar_channel(axis=axis, flow=flow), prec)
    run(inp.tilted_channel(steps=0), prec)
    run(inp.force_poiseuille(n=12, tau=0.9, force=1e-5, other=5), prec)
with lbm.Batch(4, "f32") as b:
    lats = [lbm.Lattice.from_workload(w, "f32") for w in
            (inp.couette(), inp.pillar_channel(), inp.duct(37, 19, 23, 0.8, 0.05, 30.0))]
    for i, lat in enumerate(lats):
        b.attach(i, lat)
    b.step(6, residual=True)
    b.step(3)
    for lat in lats:
        lat.close()
ran.append(("batch", "f32", "ab"))
for prec in ("f32", "f16"):
    with lbm.Batch(4, prec) as b:                   # AA lattices: both batched AA steps
        lats = [lbm.Lattice.from_workload(w, prec, scheme="aa") for w in
                (inp.duct(37, 19, 23, 0.8, 0.05, 30.0), inp.channel(33, 20, 21, 0.7, (0.04, 0.01, 0.0)),
                 inp.random_pressure_workload(28, 13, 10, 11, 0.9), inp.couette())]
        for i, lat in enumerate(lats):
            b.attach(i, lat)
        b.step(10, residual=True)
        b.step(4)
        for lat in lats:
            lat.close()
    ran.append(("batch", prec, "aa"))
enabled, count = debug_bounds_errors()
print(json.dumps({"enabled": enabled, "count": count, "lattices": len(ran)}))
"""


def test_no_index_leaves_its_buffer():
    from paper_0811_4593_gb300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", BATTERY, ROOT], capture_output=True, text=True, env=env,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["enabled"], out
    assert out["lattices"] >= 40
    assert out["count"] == 0, out


def test_an_allocator_hook_that_returns_misaligned_memory_is_refused():
    # the sweeps read population rows with 16-byte bulk copies: a buffer that is not
    # 256-byte aligned must fail the allocation, not reach a kernel
    import ctypes as C

    import torch

    import lbm_inputs as inp
    import paper_0811_4593_gb300 as lbm
    from paper_0811_4593_gb300 import _binding as b
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    keep = []
    ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
    FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

    def _alloc(nbytes, _user):
        t = torch.empty(int(nbytes) + 1024, dtype=torch.uint8, device="cuda")
        keep.append(t)
        return t.data_ptr() + 16

    def _free(_ptr, _user):
        pass

    hooks = (ALLOC(_alloc), FREE(_free))
    prev = b._hooks
    b.check(b.lib().lbm_set_allocator(C.cast(hooks[0], C.c_void_p), C.cast(hooks[1], C.c_void_p), None))
    try:
        wl = inp.channel(256, 4, 3, 0.8, (0.04, 0.01, 0.0))
        with pytest.raises(lbm.LBMError) as e:
            lbm.Lattice.from_workload(wl, "f16", torch_allocator=False)
        assert e.value.status == -2
    finally:
        if prev is not None:
            b.check(b.lib().lbm_set_allocator(C.cast(prev[0], C.c_void_p), C.cast(prev[1], C.c_void_p), None))
        else:
            b.use_default_allocator()
