"""Pins of the oracle's solid nodes (mid-grid bounce-back, Sec. "Boundary conditions"),
CPU only: a fluid region sealed by solid nodes conserves its mass exactly, solid nodes
keep their populations, and mirroring the geometry mirrors the flow."""
import numpy as np

import lbm_inputs as inp


def sealed_box(n=8):
    solid = np.zeros((n, n, n), np.uint8)
    solid[[0, -1], :, :] = 1
    solid[:, [0, -1], :] = 1
    solid[:, :, [0, -1]] = 1
    wl = inp.make_workload("box", n, n, n, 0.7, [None] * 6)
    wl.solid = solid
    return wl


def test_sealed_fluid_conserves_mass_exactly(orc):
    wl = sealed_box()
    lat = orc.Lattice.from_workload(wl)
    f0 = orc.init_equilibrium(lat) * (1 + 0.05 * inp.noise(3, lat.shape))
    fluid = wl.solid == 0
    m0 = f0[:, fluid].sum()
    f = f0
    for _ in range(20):
        f = orc.step(lat, f)
        assert abs(f[:, fluid].sum() - m0) / m0 < 1e-14
    np.testing.assert_array_equal(f[:, wl.solid == 1], f0[:, wl.solid == 1])


def test_mirrored_tilted_channel_mirrors_the_flow(orc):
    # x -> nx - 1 - x maps the channel tilted by +40 onto the one tilted by -40
    a = inp.tilted_channel(shift=40, steps=0)
    b = inp.tilted_channel(shift=-40, steps=0)
    np.testing.assert_array_equal(a.solid[:, :, ::-1], b.solid)
    c, _, _ = orc.lattice()
    idx = {tuple(v): k for k, v in enumerate(c)}
    pi = np.array([idx[(-v[0], v[1], v[2])] for v in c])
    la, lb = orc.Lattice.from_workload(a), orc.Lattice.from_workload(b)
    fa = orc.run(la, orc.init_equilibrium(la), 40, form=1)
    fb = orc.run(lb, orc.init_equilibrium(lb), 40, form=1)
    fm = np.empty_like(fa)
    fm[pi] = fa[:, :, :, ::-1]
    np.testing.assert_allclose(fm, fb, rtol=0, atol=1e-15)


def test_inflow_plane_carries_the_prescribed_profile(orc):
    wl = inp.tilted_channel(steps=0)
    lat = orc.Lattice.from_workload(wl)
    f = orc.run(lat, orc.init_equilibrium(lat), 30, form=1)
    _, u = orc.macros(lat, f)
    fluid0 = wl.solid[0] == 0
    np.testing.assert_allclose(u[:, 0][:, fluid0].T, wl.utabs[4][fluid0], rtol=0, atol=1e-16)


def test_normal_only_inflow_readings():
    # the comparison inflow restricted to the plane normal: the profile's z component,
    # or its full speed along z; both with no tangential part, same nodes as the tilted one
    full = inp.tilted_channel(steps=0)
    comp = inp.tilted_channel(steps=0, normal_only=True)
    mag = inp.tilted_channel(steps=0, normal_only="magnitude")
    for fc in (4, 5):
        t, c, m = full.utabs[fc], comp.utabs[fc], mag.utabs[fc]
        assert not c[..., :2].any() and not m[..., :2].any()
        np.testing.assert_array_equal(c[..., 2], t[..., 2])
        np.testing.assert_allclose(m[..., 2], np.sqrt((t ** 2).sum(-1)), rtol=1e-15, atol=0)
        assert (m[..., 2] >= c[..., 2]).all() and (m[..., 2] > c[..., 2]).any()
