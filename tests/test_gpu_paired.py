"""GPU tests of the paired binary16 sweeps (two neighbouring nodes per thread).

Plain A/B steps of a binary16 lattice with an even nx run a paired sweep: the
row-staged one (whole rows copied to shared memory by bulk copies) when nx is a
multiple of 8 and at least 256, else the register-staged one; residual steps, odd nx,
geometries and forces run the single-node sweep. All apply the same per-node code, so a
lattice advanced by plain steps must hold exactly the bits of the same lattice advanced
by residual steps, and it must match the FP64 oracle within the binary16 bar.
"""
import numpy as np
import pytest

import lbm_inputs as inp
from lbm_testlib import decode, encode, noisy_state, run_pair, velocity_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)


WORKLOADS = {
    # walled x: node A of the first pair and node B of the last pair are face nodes
    "channel": lambda: inp.channel(32, 20, 21, 0.7, (0.04, 0.01, 0.0)),
    "duct": lambda: inp.duct(64, 16, 16, 0.8, 0.05, 30.0),
    "random_faces": lambda: inp.random_face_workload(7, 10, 9, 7, 1.1, (False, False, False)),
    "pressure": lambda: inp.random_pressure_workload(28, 12, 10, 11, 0.9),
    # periodic x: the first and last pairs wrap
    "periodic": lambda: inp.make_workload("periodic", 10, 7, 5, 0.6, [None] * 6),
    "couette": lambda: inp.couette(),
    "smallest": lambda: inp.random_face_workload(29, 4, 3, 3, 1.0, (False, False, False)),
    # rows of 256 or more nodes that are whole 16-byte multiples: the row-staged sweep
    "rows_channel": lambda: inp.channel(256, 6, 5, 0.7, (0.04, 0.01, 0.0)),
    "rows_duct": lambda: inp.duct(264, 9, 7, 0.8, 0.05, 30.0),
    "rows_xper": lambda: inp.random_face_workload(31, 512, 4, 5, 1.2, (True, False, False)),
    "rows_all_periodic": lambda: inp.make_workload("periodic", 256, 3, 4, 0.6, [None] * 6),
    # pressure planes at x = 0 and x = nx - 1, random velocity tables on every other face
    # (faces, edges and corners of both kinds inside the staged rows)
    "rows_pressure": lambda: inp.random_pressure_workload(32, 272, 5, 4, 0.9),
    "rows_random_faces": lambda: inp.random_face_workload(33, 264, 4, 5, 1.1, (False, False, False)),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_paired_sweep_equals_single_node_sweep(name):
    import paper_0811_4593_gb300 as lbm
    wl = WORKLOADS[name]()
    assert wl.nx % 2 == 0
    s0 = encode(noisy_state((19, wl.nz, wl.ny, wl.nx), 3, u=(0.01, -0.004, 0.006)), "f16")
    with lbm.Lattice.from_workload(wl, "f16") as a, lbm.Lattice.from_workload(wl, "f16") as b:
        a.set_populations(s0)
        b.set_populations(s0)
        launches = a.info()["kernel_launches"]
        a.step(12)                       # paired sweep
        for _ in range(12):
            b.step_residual(1)           # single-node sweep with the fused reductions
        assert a.info()["kernel_launches"] - launches == 12
        np.testing.assert_array_equal(a.get_populations(), b.get_populations())


# binary16 bars at about twice the measured velocity error (GB300: 3.9e-4, 2.4e-4, 3.9e-4,
# 3.3e-4, 4.9e-4, 3.1e-4, 3.5e-4)
PAIRED_F16_TOL = {"channel": 8e-4, "pressure": 5e-4, "periodic": 8e-4, "rows_channel": 7e-4, "rows_xper": 1e-3,
                  "rows_pressure": 7e-4, "rows_random_faces": 7e-4}


@pytest.mark.parametrize("name", list(PAIRED_F16_TOL))
def test_paired_sweep_matches_oracle(name):
    wl = WORKLOADS[name]()
    f0 = noisy_state((19, wl.nz, wl.ny, wl.nx), 9, u=(0.01, -0.004, 0.006))
    got, ref = run_pair(wl, "f16", f0, 30)
    assert velocity_error(wl, got, ref) <= PAIRED_F16_TOL[name]
    assert np.isfinite(decode(encode(got, "f16"), "f16")).all()


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_paired_aa_steps_equal_ab_steps(name):
    # the paired sweep also runs both AA steps of an even-nx binary16 lattice; the AA
    # lattice must hold the A/B lattice's bits after every pair of steps
    import paper_0811_4593_gb300 as lbm
    wl = WORKLOADS[name]()
    s0 = encode(noisy_state((19, wl.nz, wl.ny, wl.nx), 4, u=(0.01, -0.004, 0.006)), "f16")
    with lbm.Lattice.from_workload(wl, "f16") as ab, lbm.Lattice.from_workload(wl, "f16", scheme="aa") as aa:
        ab.set_populations(s0)
        aa.set_populations(s0)
        for n in (2, 6):
            ab.step(n)
            aa.step(n)
            np.testing.assert_array_equal(aa.get_populations(), ab.get_populations())
        assert aa.step_residual(2) == ab.step_residual(2)
