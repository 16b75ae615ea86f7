"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs, element by element, plus invariants at the benchmark's full size.

Tolerances (max over all nodes):
  f64  populations and velocity within 1e-12 relative;
  f32  velocity within 1e-5 of the largest velocity magnitude;
  f16  (binary16 storage of f - w rho0) velocity within F16_TOL[case] of the largest
       velocity magnitude: about twice the error measured for each case at the step
       counts used here, so that a regression of the binary16 path shows.
"""
import numpy as np
import pytest

import lbm_inputs as inp
from lbm_testlib import (decode, encode, noisy_state, population_error, run_pair, separable_state_slab,
                         separable_value_at, velocity_error)

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
# measured (GB300): couette 2.8e-4, duct_ragged 3.0e-4, channel_ragged 3.9e-4,
# random_walls 1.9e-4, random_xper 3.4e-4, random_zper 2.0e-4, periodic 4.7e-4,
# minimum_3x3x3 2.4e-4, pressure_duct_ragged 2.6e-4, pressure_random 1.6e-4,
# pressure_random_yper 2.0e-4
F16_TOL = {"couette": 6e-4, "duct_ragged": 6e-4, "channel_ragged": 8e-4, "random_walls": 4e-4,
           "random_xper": 7e-4, "random_zper": 4e-4, "periodic": 1e-3, "minimum_3x3x3": 5e-4,
           "pressure_duct_ragged": 6e-4, "pressure_random": 4e-4, "pressure_random_yper": 4e-4}
# binary16 storage in the 5000-step Couette flow from rest (measured 1.38e-2): the
# slow diffusive transient integrates the storage rounding
F16_COUETTE_5000_TOL = 2.5e-2


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def case(name):
    """Small workloads that span several 256-node blocks with a ragged tail and cover
    every node class (faces with tangential velocity, edges, corners, periodic wrap)."""
    if name == "couette":
        return inp.couette(), 60
    if name == "duct_ragged":
        return inp.duct(37, 19, 23, 0.8, 0.05, 30.0), 40
    if name == "channel_ragged":
        return inp.channel(33, 20, 21, 0.8, (0.04, 0.01, 0.0)), 40
    if name == "random_walls":
        return inp.random_face_workload(21, 11, 9, 7, 0.9, (False, False, False)), 25
    if name == "random_xper":
        return inp.random_face_workload(22, 10, 13, 6, 0.7, (True, False, False)), 25
    if name == "random_zper":
        return inp.random_face_workload(23, 12, 5, 9, 1.3, (False, False, True)), 25
    if name == "periodic":
        return inp.make_workload("periodic", 9, 7, 5, 0.6, [None] * 6), 30
    if name == "minimum_3x3x3":
        return inp.random_face_workload(24, 3, 3, 3, 1.0, (False, False, False)), 20
    if name == "pressure_duct_ragged":
        return inp.pressure_duct(9, 23, 0.8, 1.006, 0.994), 40
    if name == "pressure_random":
        return inp.random_pressure_workload(25, 13, 10, 11, 0.9), 25
    if name == "pressure_random_yper":
        return inp.random_pressure_workload(26, 12, 9, 7, 1.1, periodic_y=True), 25
    raise KeyError(name)


CASES = ["couette", "duct_ragged", "channel_ragged", "random_walls", "random_xper", "random_zper", "periodic",
         "minimum_3x3x3", "pressure_duct_ragged", "pressure_random", "pressure_random_yper"]


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("name", CASES)
def test_parity_with_oracle(name, prec):
    wl, steps = case(name)
    f0 = noisy_state((19, wl.nz, wl.ny, wl.nx), seed=100 + CASES.index(name), amp=0.02, u=(0.01, -0.005, 0.008))
    got, ref = run_pair(wl, prec, f0, steps)
    ev = velocity_error(wl, got, ref)
    tol = F16_TOL[name] if prec == "f16" else TOL[prec]
    assert ev <= tol, f"{name} {prec}: velocity error {ev:.3e}"
    if prec == "f64":
        assert population_error(got, ref) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_couette_5000_steps_against_oracle(prec):
    # BASELINE configuration 1 as stated: 5000 steps from rest, velocity error against
    # the oracle's run in units of the wall speed
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = inp.couette()
    olat = oracle.Lattice.from_workload(wl)
    ref = oracle.run(olat, oracle.init_equilibrium(olat), wl.steps)
    _, uo = oracle.macros(olat, ref)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.step(wl.steps)
        _, u = lat.macros()
        u = u.double().cpu().numpy()
    err = np.abs(u - uo).max() / np.abs(uo).max()
    assert err <= {"f64": 1e-12, "f32": 1e-5, "f16": F16_COUETTE_5000_TOL}[prec], err


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_couette_linear_profile_on_gpu(prec):
    import paper_0811_4593_gb300 as lbm
    wl = inp.couette()
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.step(wl.steps)
        _, u = lat.macros()
        u = u.double().cpu().numpy()
    z = np.arange(wl.nz)[:, None, None]
    err = np.abs(u[0] - 0.05 * z / 16).max()
    assert err < (1e-13 if prec == "f64" else 5e-7), err
    assert np.abs(u[1:]).max() < (1e-13 if prec == "f64" else 5e-7)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_population_roundtrip_and_zero_steps(prec):
    import paper_0811_4593_gb300 as lbm
    wl = inp.duct(11, 6, 7, 0.8, 0.05, 30.0)
    s0 = encode(noisy_state((19, 7, 6, 11), 5), prec)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(s0)
        lat.step(0)
        np.testing.assert_array_equal(lat.get_populations(), s0)
        # slab round trip: planes 2..4 only
        part = lat.get_populations(2, 3)
        np.testing.assert_array_equal(part, s0[:, 2:5])
        lat.set_populations(s0[:, 2:5] * 0 + s0[:, 2:5], z0=2)
        np.testing.assert_array_equal(lat.get_populations(), s0)
        assert lat.info()["steps"] == 0


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_initial_state_is_rest_equilibrium(prec):
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = inp.channel(9, 5, 6, 0.8)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        got = decode(lat.get_populations(), prec)
    ref = oracle.init_equilibrium(oracle.Lattice.from_workload(wl))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-7 if prec != "f64" else 0)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_macros_match_oracle(prec):
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = inp.duct(13, 8, 6, 0.8, 0.05, 30.0)
    s0 = encode(noisy_state((19, 6, 8, 13), 11, u=(0.02, 0.01, -0.01)), prec)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(s0)
        rho, u = lat.macros()
        rho, u = rho.double().cpu().numpy(), u.double().cpu().numpy()
    rref, uref = oracle.macros(oracle.Lattice.from_workload(wl), decode(s0, prec))
    tol = 1e-14 if prec == "f64" else 1e-6
    np.testing.assert_allclose(rho, rref, rtol=0, atol=tol)
    np.testing.assert_allclose(u, uref, rtol=0, atol=tol)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_residual_and_mass_match_oracle(prec):
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = inp.duct(19, 9, 8, 0.9, 0.05, 30.0)
    olat = oracle.Lattice.from_workload(wl)
    f0 = noisy_state((19, 8, 9, 19), 17)
    s0 = encode(f0, prec)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(s0)
        r1, m1 = lat.step_residual(10)
        r2, m2 = lat.step_residual(10)
        r3, m3 = lat.residual()
    a = oracle.run(olat, decode(s0, prec), 10)
    b = oracle.run(olat, a, 10)
    _, ua = oracle.macros(olat, a)
    red_a = oracle.reduce(olat, a, None)
    red_b = oracle.reduce(olat, b, ua)
    rtol = 1e-12 if prec == "f64" else 1e-5
    assert abs(m1 - red_a[0]) / red_a[0] < rtol
    assert abs(m2 - red_b[0]) / red_b[0] < rtol
    assert abs(r1 - 1.0) < 1e-12  # first evaluation compares with the zero snapshot
    r_ref = np.sqrt(red_b[1]) / np.sqrt(red_b[2])
    assert abs(r2 - r_ref) / r_ref < (1e-9 if prec == "f64" else 2e-3)
    assert r3 < 1e-5 and abs(m3 - m2) / m2 < rtol  # same state: snapshot just taken


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_state_residual_matches_oracle_reduce(prec):
    # lbm_residual on two stored states in a row: its mass and residual equal the
    # oracle's reduction of the same decoded populations, with u_prev the oracle's
    # velocities of the first state (so only the reduction is compared, not a run)
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = inp.duct(37, 19, 23, 0.8, 0.05, 30.0)   # 16,169 nodes: 64 blocks, ragged tail
    olat = oracle.Lattice.from_workload(wl)
    shape = (19, wl.nz, wl.ny, wl.nx)
    s0 = encode(noisy_state(shape, 61, u=(0.02, 0.01, 0.0)), prec)
    s1 = encode(noisy_state(shape, 62, u=(0.015, 0.012, -0.004)), prec)
    rtol = 1e-12 if prec == "f64" else 1e-5
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(s0)
        r0, m0 = lat.residual()
        lat.set_populations(s1)
        r1, m1 = lat.residual()
    f0, f1 = decode(s0, prec), decode(s1, prec)
    red0 = oracle.reduce(olat, f0, None)
    _, u0 = oracle.macros(olat, f0)
    red1 = oracle.reduce(olat, f1, u0)
    # the residual is a velocity difference in units of the velocity magnitude, so its
    # bar is absolute
    assert r0 == pytest.approx(np.sqrt(red0[1]) / np.sqrt(red0[2]), abs=1e-12)
    assert m0 == pytest.approx(red0[0], rel=rtol)
    assert abs(r1 - np.sqrt(red1[1]) / np.sqrt(red1[2])) <= rtol
    assert m1 == pytest.approx(red1[0], rel=rtol)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_fused_residual_matches_oracle_reduce(prec):
    # lbm_step_residual reduces inside the sweep; its sums equal the oracle's reduction
    # of the state the step stored, with u_prev the oracle's velocities of the state
    # of the previous residual step. Binary16 rounds the stored state after the
    # reduction has seen the unrounded values, so its bar is wider.
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = inp.duct(37, 19, 23, 0.8, 0.05, 30.0)
    olat = oracle.Lattice.from_workload(wl)
    s0 = encode(noisy_state((19, wl.nz, wl.ny, wl.nx), 63, u=(0.02, 0.01, 0.0)), prec)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(s0)
        r1, m1 = lat.step_residual(10)
        a = decode(lat.get_populations(), prec)
        r2, m2 = lat.step_residual(10)
        b = decode(lat.get_populations(), prec)
    _, ua = oracle.macros(olat, a)
    red_a = oracle.reduce(olat, a, None)
    red_b = oracle.reduce(olat, b, ua)
    rtol_m = 1e-12 if prec == "f64" else 1e-5
    bar_r = {"f64": 1e-12, "f32": 1e-5, "f16": 1e-3}[prec]   # absolute, in units of |u|
    assert r1 == pytest.approx(1.0, abs=1e-12)
    assert m1 == pytest.approx(red_a[0], rel=rtol_m)
    assert m2 == pytest.approx(red_b[0], rel=rtol_m)
    assert abs(r2 - np.sqrt(red_b[1]) / np.sqrt(red_b[2])) <= bar_r


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_boundary_velocity_exact_on_gpu(prec):
    import paper_0811_4593_gb300 as lbm
    wl = inp.random_face_workload(31, 10, 8, 9, 0.8, (False, False, False))
    s0 = encode(noisy_state((19, 9, 8, 10), 31), prec)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(s0)
        lat.step(7)
        _, u = lat.macros()
        u = u.double().cpu().numpy()
    tol = 1e-15 if prec == "f64" else 1e-7
    # faces (excluding edges/corners)
    x0 = u[:, 1:-1, 1:-1, 0]
    np.testing.assert_allclose(x0, wl.utabs[0][1:-1, 1:-1].transpose(2, 0, 1), rtol=0, atol=tol)
    z1 = u[:, -1, 1:-1, 1:-1]
    np.testing.assert_allclose(z1, wl.utabs[5][1:-1, 1:-1].transpose(2, 0, 1), rtol=0, atol=tol)
    # edges and corners: no slip
    for e in (u[:, 0, 0, :], u[:, -1, :, -1], u[:, :, 0, 0], u[:, 0, -1, -1]):
        np.testing.assert_allclose(e, 0, atol=tol)


def test_runs_are_bitwise_deterministic():
    import paper_0811_4593_gb300 as lbm
    wl = inp.duct(45, 17, 13, 0.7, 0.05, 30.0)
    outs = []
    for _ in range(2):
        with lbm.Lattice.from_workload(wl, "f32") as lat:
            r, m = lat.step_residual(30)
            outs.append((lat.get_populations(), r, m))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]


def test_divergence_is_reported():
    # At tau = 0.55 the no-slip face closure amplifies perturbations on this slab (the
    # oracle shows the same growth); the residual check must report it.
    import paper_0811_4593_gb300 as lbm
    wl = inp.make_workload("slab", 8, 10, 10, 0.55, [None, None, None, None, inp.ZERO, inp.ZERO])
    s0 = encode(noisy_state((19, 10, 10, 8), 3, amp=1e-3), "f32")
    with lbm.Lattice.from_workload(wl, "f32") as lat:
        lat.set_populations(s0)
        with pytest.raises(lbm.LBMDiverged):
            for _ in range(40):
                lat.step_residual(250)
    wl6 = inp.make_workload("slab", 8, 10, 10, 0.6, [None, None, None, None, inp.ZERO, inp.ZERO])
    with lbm.Lattice.from_workload(wl6, "f32") as lat:
        lat.set_populations(s0)
        for _ in range(12):
            r, _ = lat.step_residual(250)
        assert np.isfinite(r)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_pressure_planes_hold_their_density_on_gpu(prec):
    import paper_0811_4593_gb300 as lbm
    wl = inp.random_pressure_workload(27, 10, 8, 9, 0.8)
    s0 = encode(noisy_state((19, 9, 8, 10), 27), prec)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(s0)
        lat.step(6)
        rho, u = lat.macros()
        rho, u = rho.double().cpu().numpy(), u.double().cpu().numpy()
    tol = 1e-14 if prec == "f64" else 2e-7
    # x faces incl. their edges and corners carry the prescribed density
    np.testing.assert_allclose(rho[:, :, 0], wl.ptabs[0], rtol=0, atol=tol)
    np.testing.assert_allclose(rho[:, :, -1], wl.ptabs[1], rtol=0, atol=tol)
    # tangential velocity on the pressure faces (without edges/corners)
    np.testing.assert_allclose(u[1:, 1:-1, 1:-1, 0], wl.utabs[0][1:-1, 1:-1, 1:].transpose(2, 0, 1), rtol=0,
                               atol=tol)


@pytest.mark.parametrize("prec", ["f64"])
def test_pressure_duct_second_order_on_gpu(prec):
    # The paper's square-channel study: the error against eq. squarechannel falls with
    # slope ~2 in the lattice width. Like the paper, which fits only the smaller sizes
    # because at 64 nodes another error dominates, the fit uses widths 8, 16 and 32
    # (at width 64 the error levels off near 4e-4: compressibility at Mach ~0.04).
    import paper_0811_4593_gb300 as lbm

    def series(n, terms=50):
        b = n - 1.0
        s = np.arange(n) - (n - 1) / 2.0
        X, Y = np.meshgrid(s, s, indexing="ij")
        C = np.zeros_like(X)
        for m in range(terms):
            k = 2 * m + 1
            C += (-1) ** m * np.cosh(k * np.pi * X / b) * np.cos(k * np.pi * Y / b) / (k ** 3 * np.cosh(k * np.pi / 2))
        return b * b / 4 - Y ** 2 - C * 8 * b * b / np.pi ** 3

    errs, widths = [], []
    for n in (9, 17, 33):
        length = 3 * n
        wl = inp.pressure_duct(n, length, 1.0, 1.002, 0.998)
        with lbm.Lattice.from_workload(wl, prec) as lat:
            lat.step(14 * n * n)
            rho, u = lat.macros()
            rho, u = rho.double().cpu().numpy(), u.double().cpu().numpy()
        xm = length // 2
        grad = (rho[:, :, xm + 1].mean() - rho[:, :, xm - 1].mean()) / 2.0 / 3.0
        eta = rho[:, :, xm].mean() * 0.5 / 3.0
        an = -grad / (2 * eta) * series(n)
        errs.append(np.sqrt(((u[0][:, :, xm] - an) ** 2).mean() / (an ** 2).mean()))
        widths.append(n - 1)
    slopes = [np.log(errs[i] / errs[i + 1]) / np.log(widths[i + 1] / widths[i]) for i in range(2)]
    print("pressure duct errors", errs, "slopes", slopes)
    assert all(1.7 < s < 2.3 for s in slopes), (errs, slopes)


# ---------------------------------------------------------------------------------
# Full size: the 512^3 channel of the benchmark, in the benchmark's launch
# configuration, checked node by node after one step from a seeded state.
# ---------------------------------------------------------------------------------

def _sample_nodes(nx, ny, nz, planes, seed=5):
    rng_u = inp.uniform(seed, 77, np.arange(4000))
    nodes = []
    for j, z in enumerate(planes):
        xs = (rng_u[j * 400:(j * 400) + 200] * nx).astype(int)
        ys = (rng_u[j * 400 + 200:(j + 1) * 400] * ny).astype(int)
        nodes += [(x, y, z) for x, y in zip(xs, ys)]
        for y in (0, 1, ny // 2, ny - 1):
            nodes += [(0, y, z), (1, y, z), (nx - 2, y, z), (nx - 1, y, z)]
    return np.array(sorted({(z * ny + y) * nx + x for x, y, z in nodes}), np.int64)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_full_size_channel_one_step_sampled(prec):
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = inp.channel(512, 512, 512, 0.8, (0.04, 0.01, 0.0))
    nx, ny, nz = wl.dims
    amp = 0.02
    tables = inp.separable_noise_tables(1234, nx, ny, nz)
    planes = [0, 1, 255, 510, 511]
    nodes = _sample_nodes(nx, ny, nz, planes)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        for z0 in range(0, nz, 32):
            lat.set_populations(separable_state_slab(tables, nx, ny, z0, z0 + 32, amp, prec), z0=z0)
        lat.step(1)
        got = {z: decode(lat.get_populations(z, 1), prec)[:, 0] for z in planes}
    olat = oracle.Lattice.from_workload(wl)
    ref = oracle.step_nodes(olat, lambda idx: separable_value_at(tables, nx, ny, nz, idx, amp, prec), nodes)
    x = nodes % nx
    y = (nodes // nx) % ny
    z = nodes // (nx * ny)
    g = np.stack([got[int(zz)][:, yy, xx] for xx, yy, zz in zip(x, y, z)])
    tol = {"f64": 1e-13, "f32": 2e-6, "f16": 2e-5}[prec]
    assert np.abs(g - ref).max() < tol, np.abs(g - ref).max()


def test_full_size_channel_invariants_after_many_steps():
    import paper_0811_4593_gb300 as lbm
    wl = inp.channel(512, 512, 512, 0.8, (0.04, 0.01, 0.0))
    with lbm.Lattice.from_workload(wl, "f32") as lat:
        lat.step(150)
        r, m = lat.step_residual(50)
        rho, u = lat.macros()
        walls = u[:, [0, -1], :, :].abs().max().item()
        inlet = u[:, 1:-1, :, 0].double().cpu().numpy()
        outlet = u[:, 1:-1, :, -1].double().cpu().numpy()
    assert np.isfinite(r) and np.isfinite(m)
    assert walls < 2e-7
    want = np.array([0.04, 0.01, 0.0])[:, None, None]
    assert np.abs(inlet - want).max() < 2e-7
    assert np.abs(outlet - want).max() < 2e-7


def test_fp32_low_viscosity_duct_within_bar():
    # tau = 0.6: the flow relaxes slowly, so a per-step momentum bias of the float
    # collision would accumulate; FP32 must stay within 1e-5 of u_max of the oracle
    import oracle
    import paper_0811_4593_gb300 as lbm
    wl = inp.duct(128, 48, 48, 0.6, 0.05, 30.0)
    steps = 4000
    with lbm.Lattice.from_workload(wl, "f32") as lat:
        lat.step(steps)
        got = decode(lat.get_populations(), "f32")
    olat = oracle.Lattice.from_workload(wl)
    ref = oracle.run(olat, oracle.init_equilibrium(olat), steps)
    err = velocity_error(wl, got, ref)
    print("fp32 duct tau 0.6 velocity error", err)
    assert err <= 1e-5, err


@pytest.mark.parametrize("prec,tau", [("f64", 1.0), ("f64", 2.0), ("f32", 1.0)])
def test_paper_shear_32_cubed_is_linear(prec, tau):
    # the paper's shear test at its size: 32^3, x and y periodic, planes z = 0 and 31
    # moving with -0.02 and +0.02; a linear profile to rounding
    import paper_0811_4593_gb300 as lbm
    wl = inp.shear(32, 32, 32, tau, 0.02)
    nu = (tau - 0.5) / 3.0
    steps = int(36.0 * 31 ** 2 / (np.pi ** 2 * nu)) + 1
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.step(steps)
        _, u = lat.macros()
        u = u.double().cpu().numpy()
    z = np.arange(32)[:, None, None]
    err = np.abs(u[0] - (-0.02 + 0.04 * z / 31)).max() / 0.02
    print("shear 32^3", prec, tau, err)
    # FP32: a steady flow integrates its per-step rounding over its relaxation time
    # (~580 steps here); measured 5.5e-6 of the wall speed
    assert err < (1e-12 if prec == "f64" else 1e-5), err
