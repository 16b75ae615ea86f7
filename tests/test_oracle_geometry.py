"""Pins of the oracle's solid nodes (mid-grid bounce-back, Sec. "Boundary conditions"),
CPU only: a fluid region sealed by solid nodes conserves its mass exactly, solid nodes
keep their populations, mirroring the geometry mirrors the flow, and the tilted channel
gives the paper's error measure."""
import numpy as np
import pytest

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


@pytest.mark.slow
def test_tilted_channel_xi_against_the_paper(orc):
    # The paper's tilted-channel table: xi = 0.0996 for the on-site inflow, 0.175 with
    # the inflow restricted to the plane normal, 0.00235 for the straight channel. With
    # its averaging volume and wall position read as stated in the tilted-channel
    # workload (all fluid nodes; fluid where |x - x_c(z)| < 10), the on-site value is
    # matched within 10 %, the normal-only inflow is clearly worse under either reading
    # of its normal velocity, and the straight channel stays below the paper's value.
    # 3000 steps: the relaxation time across the channel (20^2 / (pi^2 nu)) is ~240 steps.
    import bench

    def xi(wl, ref):
        lat = orc.Lattice.from_workload(wl)
        _, u = orc.macros(lat, orc.run(lat, orc.init_equilibrium(lat), 3000))
        return bench.tilted_xi(ref, u)

    tilted = inp.tilted_channel()
    on_site = xi(tilted, tilted)
    assert abs(on_site / 0.0996 - 1) < 0.10
    for reading in (True, "magnitude"):
        assert xi(inp.tilted_channel(normal_only=reading), tilted) > 1.15 * on_site
    straight = inp.tilted_channel(shift=0)
    assert xi(straight, straight) < 0.00235
