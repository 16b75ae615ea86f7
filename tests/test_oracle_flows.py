"""Whole-lattice pins of the oracle (CPU only): closed-form flows, invariants that
hold at any size, and symmetry of the complete time step.
"""
import numpy as np
import pytest

import lbm_inputs as inp

Z = inp.ZERO


def boundary_masks(wl):
    """Boolean masks (face[6], edge, corner) over [nz][ny][nx]."""
    z, y, x = np.meshgrid(np.arange(wl.nz), np.arange(wl.ny), np.arange(wl.nx), indexing="ij")
    coords = (x, y, z)
    dims = wl.dims
    on = []
    for a in range(3):
        walled = wl.kinds[2 * a] == inp.VELOCITY
        on.append((walled & (coords[a] == 0), walled & (coords[a] == dims[a] - 1)))
    count = sum(lo.astype(int) + hi.astype(int) for lo, hi in on)
    faces = [on[f // 2][f % 2] & (count == 1) for f in range(6)]
    return faces, count == 2, count == 3


def noisy_state(orc, lat, seed, amp=0.02, u=(0.01, -0.005, 0.008)):
    base = orc.feq(1.0, u)
    return base[:, None, None, None] * (1 + amp * inp.noise(seed, lat.shape))


def test_couette_is_linear_to_rounding(orc):
    # Shear between a resting wall at z=0 and a wall moving with 0.05 at z=16 settles
    # to u_x = 0.05 z / 16 (the paper: linear within floating-point precision).
    wl = inp.couette()
    lat = orc.Lattice.from_workload(wl)
    f = orc.run(lat, orc.init_equilibrium(lat), wl.steps)
    rho, u = orc.macros(lat, f)
    z = np.arange(wl.nz)[:, None, None]
    assert np.abs(u[0] - 0.05 * z / 16).max() < 1e-13
    assert np.abs(u[1]).max() < 1e-13 and np.abs(u[2]).max() < 1e-13
    # closed walls: steady mass is conserved to rounding
    m0 = orc.reduce(lat, f)[0]
    m1 = orc.reduce(lat, orc.step(lat, f))[0]
    assert abs(m1 - m0) / m0 < 1e-14


@pytest.mark.parametrize("tau", [1.0, 2.0, 0.7])
def test_opposite_wall_shear_is_linear_to_rounding(orc, tau):
    # The paper's shear test: planes z = 0 and z = 31 moving with -0.02 and +0.02 along x,
    # periodic x and y (4 x 4 nodes suffice for the one-dimensional flow); the profile is
    # u_x = -0.02 + 0.04 z / 31 to rounding, for any tau.
    wl = inp.shear(4, 4, 32, tau, 0.02)
    lat = orc.Lattice.from_workload(wl)
    nu = (tau - 0.5) / 3.0
    steps = int(36.0 * 31 ** 2 / (np.pi ** 2 * nu)) + 1   # slowest mode below e^-36
    f = orc.run(lat, orc.init_equilibrium(lat), steps)
    _, u = orc.macros(lat, f)
    z = np.arange(wl.nz)[:, None, None]
    assert np.abs(u[0] - (-0.02 + 0.04 * z / 31)).max() < 1e-14
    assert np.abs(u[1]).max() < 1e-14 and np.abs(u[2]).max() < 1e-14


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.5])
@pytest.mark.parametrize("periodic", [(False, False, False), (False, True, False), (True, False, True)])
def test_boundary_velocity_is_exact_after_every_step(orc, periodic, tau):
    # Face nodes carry exactly their prescribed velocity, edges and corners exactly
    # zero, after streaming, closure and collision, whatever tau (the closure does not
    # depend on it, and the wall is on the node).
    wl = inp.random_face_workload(3, 7, 6, 5, tau, periodic)
    lat = orc.Lattice.from_workload(wl)
    faces, edge, corner = boundary_masks(wl)
    f = noisy_state(orc, lat, 5)
    for _ in range(6):
        f = orc.step(lat, f)
        _, u = orc.macros(lat, f)
        for fc in range(6):
            if not faces[fc].any():
                continue
            tab = wl.utabs[fc]
            a = fc // 2
            t1, t2 = [b for b in range(3) if b != a]
            zz, yy, xx = np.nonzero(faces[fc])
            c = (xx, yy, zz)
            want = tab[c[t2], c[t1]]
            got = u[:, zz, yy, xx].T
            np.testing.assert_allclose(got, want, rtol=0, atol=2e-16)
        np.testing.assert_allclose(u[:, edge | corner], 0, atol=2e-16)


def _permute_workload(wl, perm):
    """Relabel axes: new axis i is old axis perm[i] (dims, tables and vectors)."""
    dims = [wl.dims[p] for p in perm]
    face_u = [None] * 6
    for nf in range(6):
        na, side = nf // 2, nf % 2
        tab = wl.utabs[2 * perm[na] + side]
        if tab is None:
            continue
        old_t1 = min(b for b in range(3) if b != perm[na])
        new_t1 = min(b for b in range(3) if b != na)
        # tables are indexed [t2][t1]; transpose when the new t1 is the old t2
        arr = tab if perm[new_t1] == old_t1 else np.transpose(tab, (1, 0, 2))
        face_u[nf] = np.ascontiguousarray(arr[..., list(perm)])
    return inp.make_workload("perm", *dims, wl.tau, face_u)


def test_axis_permutation_symmetry_of_full_steps(orc):
    # The time step commutes with relabelling the axes: all face, edge and corner
    # rules of one orientation are checked against the others.
    wl = inp.random_face_workload(8, 7, 5, 6, 0.9, (False, False, False))
    lat = orc.Lattice.from_workload(wl)
    c, _, _ = orc.lattice()
    f = noisy_state(orc, lat, 9)
    g = orc.run(lat, f, 12)
    for perm in [(2, 0, 1), (1, 2, 0), (0, 2, 1), (2, 1, 0)]:
        wp = _permute_workload(wl, perm)
        lp = orc.Lattice.from_workload(wp)
        idx = {tuple(v): k for k, v in enumerate(c)}
        pi = np.array([idx[tuple(c[k][list(perm)])] for k in range(19)])
        # node arrays are [z][y][x] = axes (2,1,0); new axis i is old axis perm[i]
        ax = [2 - perm[2 - j] for j in range(3)]
        fp = np.empty(lp.shape)
        fp[pi] = np.transpose(f, [0] + [1 + a for a in ax])
        gp = orc.run(lp, fp, 12)
        np.testing.assert_allclose(gp[pi], np.transpose(g, [0] + [1 + a for a in ax]), rtol=0, atol=1e-14)


def test_compact_and_explicit_forms_agree_over_many_steps(orc):
    wl = inp.random_face_workload(11, 6, 7, 5, 0.7, (False, True, False))
    lat = orc.Lattice.from_workload(wl)
    f = noisy_state(orc, lat, 12)
    g0 = orc.run(lat, f, 40, form=0)
    g1 = orc.run(lat, f, 40, form=1)
    np.testing.assert_allclose(g0, g1, rtol=0, atol=1e-14)


def test_node_sampled_step_matches_full_step(orc):
    # The node-by-node evaluation used for very large lattices is the same step.
    wl = inp.duct(13, 6, 7, 0.8, 0.05, 30.0)
    lat = orc.Lattice.from_workload(wl)
    f = noisy_state(orc, lat, 13)
    full = orc.step(lat, f)
    nodes = np.arange(lat.n)
    flat = f.reshape(-1)
    part = orc.step_nodes(lat, lambda idx: flat[idx], nodes)
    np.testing.assert_array_equal(part.T.reshape(lat.shape), full)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.5])
def test_poiseuille_zero_wall_slip_any_tau(orc, tau):
    # The wall sits exactly on the nodes, independent of tau: zero velocity there.
    wl = inp.poiseuille(lz=16, tau=tau)
    lat = orc.Lattice.from_workload(wl)
    nst = int(3 * 16 * 16 / ((tau - 0.5) / 3))
    f = orc.run(lat, orc.init_equilibrium(lat), nst)
    _, u = orc.macros(lat, f)
    assert np.abs(u[:, [0, -1]]).max() < 1e-16
    prof = 0.02 * inp.parabola(16)
    err = np.sqrt(((u[0] - prof[:, None, None]) ** 2).mean() / (prof ** 2).mean())
    assert err < 0.02


def test_poiseuille_error_falls_with_resolution(orc):
    errs = []
    for lz in (16, 32):
        wl = inp.poiseuille(lz=lz, tau=1.0)
        lat = orc.Lattice.from_workload(wl)
        f = orc.run(lat, orc.init_equilibrium(lat), 18 * lz * lz)
        _, u = orc.macros(lat, f)
        prof = 0.02 * inp.parabola(lz)
        errs.append(np.sqrt(((u[0] - prof[:, None, None]) ** 2).mean() / (prof ** 2).mean()))
    assert errs[1] < errs[0] / 2.5


def square_duct_series(n, terms=50):
    """Pressure-driven square-duct profile (eq. squarechannel) on nodes 0..n-1 with
    the walls on the end nodes, up to a constant factor."""
    b = n - 1.0
    s = np.arange(n) - (n - 1) / 2.0
    X, Y = np.meshgrid(s, s, indexing="ij")
    C = np.zeros_like(X)
    for m in range(terms):
        k = 2 * m + 1
        C += (-1) ** m * np.cosh(k * np.pi * X / b) * np.cos(k * np.pi * Y / b) / (k ** 3 * np.cosh(k * np.pi / 2))
    C *= 8 * b * b / np.pi ** 3
    return b * b / 4 - Y ** 2 - C


@pytest.mark.slow
def test_duct_develops_square_channel_profile(orc):
    # Far from the inlet the duct flow takes the analytic square-channel shape; the
    # difference falls as the cross-section is refined.
    errs = []
    for n in (9, 13):
        wl = inp.duct(nx=4 * n, ny=n, nz=n, tau=1.0, peak=0.02, angle_deg=0.0)
        lat = orc.Lattice.from_workload(wl)
        f = orc.run(lat, orc.init_equilibrium(lat), 12 * n * n)
        _, u = orc.macros(lat, f)
        mid = u[0][:, :, 2 * n]
        an = square_duct_series(n)
        an = an / an.mean() * mid.mean()
        errs.append(np.sqrt(((mid - an) ** 2).mean() / (an ** 2).mean()))
    assert errs[0] < 3e-3
    assert errs[1] < errs[0]


def test_low_tau_wall_instability_is_reproducible(orc):
    # The paper reports tau = 1 and tau = 2 only. At tau = 0.55 the no-slip face
    # closure amplifies a small perturbation on this slab (no edges, no corners);
    # at tau = 0.6 it decays. Both the oracle and the CUDA path must show this.
    def growth(tau):
        wl = inp.make_workload("slab", 8, 10, 10, tau, [None, None, None, None, Z, Z])
        lat = orc.Lattice.from_workload(wl)
        f0 = orc.init_equilibrium(lat)
        f = f0 * (1 + 1e-10 * inp.noise(1, lat.shape))
        f = orc.run(lat, f, 200)
        d1 = np.abs(f - f0).max()
        f = orc.run(lat, f, 400)
        return (np.abs(f - f0).max() / d1) ** (1 / 400)
    assert growth(0.55) > 1.01
    assert growth(0.6) < 1.0


@pytest.mark.parametrize("tau,steps", [(2.0, 4000), (1.0, 8000)])
def test_wall_slip_without_transverse_corrections_is_two_tau_f(orc, tau, steps):
    # Body-force Poiseuille (walls on the x faces, y and z periodic, F along z) with the
    # closure's transverse corrections set to zero. On a wall node of this y-z-uniform
    # flow the bounced-back diagonals cancel in the z momentum, and the in-plane
    # populations are the node's own post-collision values, relaxed towards the
    # equilibrium at (j + tau F) / rho; their z momentum is 2/3 of that equilibrium's,
    # so in the steady state j_z = (1 - 1/tau) j_z + (2/3) (j_z + tau F) / tau, i.e.
    # j_z = 2 tau F: the wall slips by 2 tau F / rho (the paper's 4e-5 at tau = 2 is
    # F = 1e-5). With the corrections the slip is zero (the exact Poiseuille pins).
    F = 1e-5
    wl = inp.force_poiseuille(n=32, tau=tau, force=F, other=3)
    lat = orc.Lattice.from_workload(wl)
    f = orc.run(lat, orc.init_equilibrium(lat), steps, form=orc.FORM_COMPACT_NO_N)
    rho, u = orc.macros(lat, f)
    # velocity after the boundary rule: the stored (post-collision) velocity minus F / rho
    slip = (u[2] - F / rho)[:, :, [0, -1]]
    np.testing.assert_allclose(slip, 2 * tau * F / rho[:, :, [0, -1]], rtol=1e-8, atol=0)


def _face_only(seed, matched):
    wl = inp.random_face_workload(seed, 7, 5, 6, 0.8, (False, True, True))
    if matched:   # the outflow plane carries the inflow plane's table
        tab = wl.utabs[0]
        wl = inp.make_workload("matched", 7, 5, 6, 0.8, [tab, tab.copy(), None, None, None, None])
    return wl


@pytest.mark.parametrize("matched", [False, True])
def test_global_mass_balance_of_in_and_outflow_planes(orc, matched):
    # Velocity planes at x = 0 and x = nx - 1, y and z periodic (no edges or corners).
    # The collision keeps mass and momentum and the pull stream only moves populations,
    # so one step changes the mass by what the closure writes on the face nodes minus
    # what streams out of the domain. Written with a face node's normal momentum
    # j.n = sum_{c.n>0} f - sum_{c.n<0} f after the closure (j = rho u with u the
    # prescribed velocity: the boundary-velocity pins) and the outgoing populations it
    # pulled from the first interior layer, while what leaves is its own outgoing
    # post-collision values:
    #   dM = sum over face nodes of [j.n + sum_{c.n<0} (f*_i(x - c_i) - f*_i(x))].
    # This fails if the stream loses or duplicates a population at a plane, if the
    # closure writes a population it can stream, or if the collision moves mass or
    # momentum. Summed over a periodic plane, the y-z offset of x - c_i drops out.
    wl = _face_only(21, matched)
    lat = orc.Lattice.from_workload(wl)
    c, _, _ = orc.lattice()
    f = noisy_state(orc, lat, 22)
    g = orc.step(lat, f)
    rho, u = orc.macros(lat, g)          # post-collision: the same rho and u as after the closure
    dm = g.sum() - f.sum()
    balance = 0.0
    for x, inner, n in ((0, 1, 1), (wl.nx - 1, wl.nx - 2, -1)):
        balance += n * (rho[:, :, x] * u[0][:, :, x]).sum()
        for i in np.flatnonzero(c[:, 0] == -n):
            balance += f[i, :, :, inner].sum() - f[i, :, :, x].sum()
    assert abs(dm) > 1e-6                # the state is far from steady: a real test
    assert abs(dm - balance) < 1e-13 * g.sum()


def test_matched_uniform_in_and_outflow_keeps_mass_and_state(orc):
    # The uniform equilibrium of the prescribed velocity is a fixed point of the whole
    # step (the transverse corrections vanish at equilibrium and the density relation
    # is exact there): matched uniform in/outflow conserves the mass to rounding.
    u0 = (0.04, 0.01, -0.02)
    wl = inp.make_workload("uniform", 7, 5, 6, 0.8, [u0, u0, None, None, None, None])
    lat = orc.Lattice.from_workload(wl)
    f0 = orc.feq(1.0, u0)[:, None, None, None] * np.ones(lat.shape)
    f = orc.run(lat, f0, 50)
    assert abs(f.sum() / f0.sum() - 1) < 1e-14
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-15)
