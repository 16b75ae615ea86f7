"""GPU tests of AA-pattern streaming (one population array, steps in pairs).

AA lattices are checked against the FP64 oracle element by element (populations,
macroscopic fields and the residual reduction after an even number of steps, from the
same stored state, with the tolerances of the A/B parity tests), for the single-node
AA steps and for the paired binary16 AA steps (even nx). The AA scheme also performs
exactly the arithmetic of the A/B scheme on the same values and only moves them
differently through memory, so after every pair of steps its state, macroscopic
fields and residuals must equal the A/B ones bit for bit; the populations it holds
take half the device memory.
"""
import numpy as np
import pytest

import lbm_inputs as inp
from lbm_testlib import decode, encode, noisy_state, population_error, velocity_error

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
    "duct": lambda: inp.duct(37, 19, 23, 0.8, 0.05, 30.0),
    "channel": lambda: inp.channel(33, 20, 21, 0.7, (0.04, 0.01, 0.0)),
    "pressure": lambda: inp.random_pressure_workload(28, 13, 10, 11, 0.9),
    "periodic": lambda: inp.make_workload("periodic", 9, 7, 5, 0.6, [None] * 6),
    "couette": lambda: inp.couette(),
    "minimum": lambda: inp.random_face_workload(29, 3, 3, 3, 1.0, (False, False, False)),
    # even nx: binary16 lattices take the paired AA steps
    "duct_even": lambda: inp.duct(36, 19, 23, 0.8, 0.05, 30.0),
    # rows of 256 nodes: binary16 lattices take the row-staged AA steps
    "duct_rows": lambda: inp.duct(256, 7, 6, 0.8, 0.05, 30.0),
}
# steps of the oracle comparison (even: an AA lattice is observable between pairs)
ORACLE_STEPS = {"duct": 40, "channel": 40, "pressure": 26, "periodic": 30, "couette": 60, "minimum": 20,
                "duct_even": 40, "duct_rows": 20}
# velocity error bars against the oracle, as in the A/B parity tests: FP64 and FP32 at
# the fixed bars, binary16 storage at about twice the error measured for each case
TOL = {"f64": 1e-12, "f32": 1e-5}
F16_TOL = {"duct": 6e-4, "channel": 8e-4, "pressure": 6e-4, "periodic": 9e-4, "couette": 3e-4, "minimum": 2e-4,
           "duct_even": 6e-4, "duct_rows": 5e-4}


def make(wl, prec, scheme, seed):
    import paper_0811_4593_gb300 as lbm
    lat = lbm.Lattice.from_workload(wl, prec, scheme=scheme)
    lat.set_populations(encode(noisy_state((19, wl.nz, wl.ny, wl.nx), seed, u=(0.01, -0.004, 0.006)), prec))
    return lat


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_aa_matches_oracle(name, prec):
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = WORKLOADS[name]()
    steps = ORACLE_STEPS[name]
    tol = F16_TOL[name] if prec == "f16" else TOL[prec]
    s0 = encode(noisy_state((19, wl.nz, wl.ny, wl.nx), 300 + list(WORKLOADS).index(name),
                            u=(0.01, -0.004, 0.006)), prec, wl.rho0)
    olat = oracle.Lattice.from_workload(wl)
    half = 2 * (steps // 4)                  # an even split of the steps
    mid = oracle.run(olat, decode(s0, prec, wl.rho0), half)
    with lbm.Lattice.from_workload(wl, prec, scheme="aa") as lat:
        assert lat.info()["scheme"] == 1
        lat.set_populations(s0)
        lat.step(half)
        got_mid = decode(lat.get_populations(), prec, wl.rho0)
        r_mid, _ = lat.residual()            # snapshot <- velocities of the mid state
        lat.step(steps - half)
        got = decode(lat.get_populations(), prec, wl.rho0)
        rho, u = lat.macros()
        rho, u = rho.double().cpu().numpy(), u.double().cpu().numpy()
        r_end, m_end = lat.residual()
    ref = oracle.run(olat, mid, steps - half)
    for g, r in ((got_mid, mid), (got, ref)):
        ev = velocity_error(wl, g, r)
        assert ev <= tol, f"{name} {prec} AA: velocity error {ev:.3e}"
        if prec == "f64":
            assert population_error(g, r) <= 1e-12
    # macroscopic fields of the AA state (read from its swapped slots) against the
    # oracle's moments of the oracle state
    rref, uref = oracle.macros(olat, ref)
    scale = np.abs(uref).max()
    assert np.abs(u - uref).max() <= tol * scale
    assert np.abs(rho - rref).max() <= (1e-12 if prec == "f64" else tol)
    # the residual reduction of the AA state against the oracle's, both on the GPU's
    # own states (so that trajectory differences do not enter). The residual is a
    # velocity difference in units of the velocity magnitude, so its bar is absolute:
    # the float snapshot of the mid state carries rounding of order 1e-7 |u|.
    assert r_mid == pytest.approx(1.0, abs=1e-12)
    _, u_mid = oracle.macros(olat, got_mid)
    red = oracle.reduce(olat, got, u_mid)
    bar = 1e-12 if prec == "f64" else 1e-5
    assert m_end == pytest.approx(red[0], rel=bar)
    assert abs(r_end - np.sqrt(red[1]) / np.sqrt(red[2])) <= bar


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_aa_equals_ab_bitwise(name, prec):
    wl = WORKLOADS[name]()
    with make(wl, prec, "ab", 5) as ab, make(wl, prec, "aa", 5) as aa:
        for n in (2, 4, 8):
            ab.step(n)
            aa.step(n)
            np.testing.assert_array_equal(aa.get_populations(), ab.get_populations())
        assert aa.step_residual(6) == ab.step_residual(6)
        rho_a, u_a = aa.macros()
        rho_b, u_b = ab.macros()
        assert (rho_a == rho_b).all() and (u_a == u_b).all()
        assert aa.residual() == ab.residual()


def test_aa_halves_the_population_memory():
    wl = inp.duct(64, 32, 32, 0.8, 0.05, 30.0)
    with make(wl, "f32", "ab", 1) as ab, make(wl, "f32", "aa", 1) as aa:
        pops = 19 * 4 * wl.cells
        assert ab.info()["device_bytes"] - aa.info()["device_bytes"] == pops
        assert aa.info()["scheme"] == 1


def test_aa_steps_in_pairs_and_is_observable_between_pairs():
    import paper_0811_4593_gb300 as lbm
    wl = inp.couette()
    with make(wl, "f32", "aa", 2) as aa:
        with pytest.raises(lbm.LBMError):
            aa.step(3)
        with pytest.raises(lbm.LBMError):
            aa.step_residual(1)
        aa.step(2)
        aa.get_populations()
        assert aa.info()["steps"] == 2


def test_aa_state_loaded_mid_run_matches_ab():
    wl = WORKLOADS["pressure"]()
    with make(wl, "f32", "ab", 7) as ab, make(wl, "f32", "aa", 8) as aa:
        ab.step(4)
        aa.step(6)
        state = ab.get_populations()
        aa.set_populations(state)     # overwrite the AA lattice with the A/B state
        ab.step(10)
        aa.step(10)
        np.testing.assert_array_equal(aa.get_populations(), ab.get_populations())


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_batched_aa_lattices_match_solo_ab(prec):
    import paper_0811_4593_gb300 as lbm
    names = ["duct", "channel", "pressure", "couette"]
    solo = []
    for i, nm in enumerate(names):
        with make(WORKLOADS[nm](), prec, "ab", 20 + i) as lat:
            lat.step(9)
            r = lat.step_residual(1)
            lat.step(10)
            solo.append((lat.get_populations(), r))
    with lbm.Batch(4, prec) as b:
        lats = [make(WORKLOADS[nm](), prec, "aa", 20 + i) for i, nm in enumerate(names)]
        for i, lat in enumerate(lats):
            b.attach(i, lat)
        with pytest.raises(lbm.LBMError):
            b.step(5)
        b.step(10, residual=True)
        res = b.results()
        b.step(10)
        for i, lat in enumerate(lats):
            np.testing.assert_array_equal(lat.get_populations(), solo[i][0])
            assert res[i][:2] == solo[i][1]
        ab_lat = make(WORKLOADS["duct"](), prec, "ab", 1)
        b.detach(0)
        with pytest.raises(lbm.LBMError):
            b.attach(0, ab_lat)           # the batch holds AA lattices
        ab_lat.close()
        for lat in lats:
            lat.close()
