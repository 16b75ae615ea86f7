"""Pins of the oracle's general-geometry rules and body force, CPU only.

Boundary nodes of a general geometry carry their normal as an integer code (Sec.
"On-site no-slip boundary condition", complex geometries): planes (eq. bbshort with
v = 0), concave edges (eq. edge), convex edges (eq. edge2), corners (eq. corner) and
junctions of a convex edge with a plane. The pins:
  * each code overwrites exactly the populations whose source lies in the solid
    region the code describes (built here from half-spaces, independently of the
    oracle's decoding);
  * plane, concave-edge and corner codes are the box rules already pinned elsewhere;
  * convex edges leave no momentum along the edge, junctions none through the plane,
    and both keep a resting equilibrium;
  * every rule commutes with the 48 symmetries of the cube;
  * walls moved into the domain as coded nodes give the box result bit for bit;
  * the body force of eq. gravity gives the exact Poiseuille parabola (eq. poiseuille
    with the viscosity of eq. visc) with zero velocity on the wall nodes;
  * the flow around a pillar is mirror-symmetric when the geometry is, and its
    boundary nodes hold the momenta the rules prescribe.
"""
import itertools

import numpy as np
import pytest

import lbm_inputs as inp

AXES = [np.array(v) for v in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]


def configurations():
    """(kind, normals, code) for every geometric configuration the codes name."""
    out = []
    for n in AXES:
        out.append(("plane", (n,), inp.plane_code(n)))
    pairs = [(a, b) for a, b in itertools.combinations(AXES, 2) if a @ b == 0 and np.any(a + b != 0)]
    for a, b in pairs:
        out.append(("concave", (a, b), inp.concave_edge_code(a, b)))
        out.append(("convex", (a, b), inp.convex_edge_code(a, b)))
    for s in itertools.product((1, -1), repeat=3):
        out.append(("corner", (np.array(s),), inp.corner_code(s)))
    for n in AXES:
        for a, b in pairs:
            if a @ n == 0 and b @ n == 0:
                out.append(("junction", (n, a, b), inp.junction_code(n, a, b)))
    return out


def solid_side(kind, normals, dx):
    """Whether offset dx from the node lies in the solid region of a configuration
    (normals point into the fluid)."""
    if kind == "plane":
        return dx @ normals[0] < 0
    if kind == "concave":
        return dx @ normals[0] < 0 or dx @ normals[1] < 0
    if kind == "convex":
        return dx @ normals[0] < 0 and dx @ normals[1] < 0
    if kind == "corner":
        s = normals[0]
        return any(dx[a] * s[a] < 0 for a in range(3))
    n, a, b = normals
    return dx @ n < 0 or (dx @ a < 0 and dx @ b < 0)


def test_codes_cover_the_encoding():
    codes = sorted(c for _, _, c in configurations())
    assert codes == sorted(list(range(-18, -6)) + list(range(1, 51)))


def test_rule_unknowns_are_the_populations_from_the_solid_side(orc):
    c, _, _ = orc.lattice()
    for kind, normals, code in configurations():
        blocked = np.array([solid_side(kind, normals, -c[k]) for k in range(19)])
        np.testing.assert_array_equal(orc.rule_unknowns(code), blocked, err_msg=f"{kind} {code}")
    counts = {"plane": 5, "concave": 9, "convex": 1, "corner": 12, "junction": 6}
    for kind, _, code in configurations():
        assert orc.rule_unknowns(code).sum() == counts[kind]


def random_state(orc, seed, u=(0.02, -0.01, 0.015)):
    return orc.feq(1.03, u) * (1.0 + 0.1 * inp.noise(seed, (19,)))


def face_of(n):
    a = int(np.flatnonzero(n)[0])
    return 2 * a + (0 if n[a] > 0 else 1)


def test_plane_edge_and_corner_codes_are_the_box_rules(orc):
    f = random_state(orc, 1)
    for kind, normals, code in configurations():
        got = orc.close_rule(code, f)
        if kind == "plane":
            ref, _ = orc.close_face(face_of(normals[0]), f, np.zeros(3))
        elif kind == "concave":
            ref = orc.close_edge(face_of(normals[0]), face_of(normals[1]), f)
        elif kind == "corner":
            s = normals[0]
            ref = orc.close_corner(0 if s[0] > 0 else 1, 2 if s[1] > 0 else 3, 4 if s[2] > 0 else 5, f)
        else:
            continue
        np.testing.assert_array_equal(got, ref, err_msg=f"{kind} {code}")


def test_convex_edge_removes_the_momentum_along_the_edge(orc):
    c, _, opp = orc.lattice()
    for kind, normals, code in configurations():
        if kind != "convex":
            continue
        a, b = normals
        d, e = a + b, np.cross(a, b)
        kd = next(k for k in range(19) if np.array_equal(c[k], d))
        for seed in range(5):
            f = random_state(orc, 10 + seed)
            g = orc.close_rule(code, f)
            assert abs(g @ (c @ e)) < 2e-16
            # bounce-back of the population from the solid side; the correction only
            # touches populations travelling into the bulk and keeps the density
            assert g[kd] == f[opp[kd]]
            bb = f.copy()
            bb[kd] = f[opp[kd]]
            assert abs(g.sum() - bb.sum()) < 1e-15
            into_bulk = (c @ d) > 0
            np.testing.assert_array_equal(g[~into_bulk], bb[~into_bulk])
        rest = orc.feq(0.97, np.zeros(3))
        np.testing.assert_allclose(orc.close_rule(code, rest), rest, rtol=0, atol=1e-17)


def test_junction_bounces_back_and_sets_the_rest_population(orc):
    c, _, opp = orc.lattice()
    for kind, normals, code in configurations():
        if kind != "junction":
            continue
        n = normals[0]
        unknown = orc.rule_unknowns(code)
        f = random_state(orc, 3)
        g = orc.close_rule(code, f)
        assert abs(g @ (c @ n)) < 2e-16          # nothing crosses the plane
        for k in np.flatnonzero(unknown):
            assert g[k] == f[opp[k]]
        keep = ~unknown
        keep[18] = False
        np.testing.assert_array_equal(g[keep], f[keep])
        assert abs(g[18] - g.sum() / 3.0) < 1e-16  # 12/36 of the node density
        for rho in (0.8, 1.0, 1.3):
            rest = orc.feq(rho, np.zeros(3))
            np.testing.assert_allclose(orc.close_rule(code, rest), rest, rtol=1e-15, atol=0)


def cube_symmetries():
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            m = np.zeros((3, 3), int)
            for i, p in enumerate(perm):
                m[i, p] = signs[i]
            mats.append(m)
    return mats


def code_of(kind, normals):
    if kind == "plane":
        return inp.plane_code(normals[0])
    if kind == "concave":
        return inp.concave_edge_code(*normals)
    if kind == "convex":
        return inp.convex_edge_code(*normals)
    if kind == "corner":
        return inp.corner_code(normals[0])
    return inp.junction_code(*normals)


def test_rules_commute_with_the_cube_symmetries(orc):
    c, _, _ = orc.lattice()
    index = {tuple(v): k for k, v in enumerate(c)}
    f = random_state(orc, 7)
    cfgs = configurations()
    for m in cube_symmetries():
        perm = np.array([index[tuple(m @ c[k])] for k in range(19)])   # k -> population of R c_k
        g = np.empty_like(f)
        g[perm] = f
        for kind, normals, code in cfgs:
            rcode = code_of(kind, tuple(m @ v for v in normals))
            want = np.empty_like(f)
            want[perm] = orc.close_rule(code, f)
            np.testing.assert_allclose(orc.close_rule(rcode, g), want, rtol=0, atol=1e-15,
                                       err_msg=f"{kind} {code} -> {rcode}")


def noisy(orc, lat, seed):
    return orc.init_equilibrium(lat) * (1.0 + 0.02 * inp.noise(seed, lat.shape))


@pytest.mark.parametrize("walls", [(False, False, True), (False, True, True), (True, True, True)])
def test_embedded_walls_equal_box_walls_bitwise(orc, walls):
    face_u = [inp.ZERO if walls[i // 2] else None for i in range(6)]
    box = inp.make_workload("box", 9, 7, 6, 0.8, face_u)
    box.force = np.array([3e-5, -1e-5, 2e-5])
    emb = inp.embedded_walls(box)
    lb, le = orc.Lattice.from_workload(box), orc.Lattice.from_workload(emb)
    assert orc.check_geometry(le) == -1
    f0 = noisy(orc, lb, 5)
    pad = emb.meta["pad"]
    inner = (slice(None), slice(pad[2], pad[2] + box.nz), slice(pad[1], pad[1] + box.ny),
             slice(pad[0], pad[0] + box.nx))
    g0 = orc.init_equilibrium(le)
    g0[inner] = f0
    fb = orc.run(lb, f0, 25)
    fe = orc.run(le, g0, 25)
    np.testing.assert_array_equal(fe[inner], fb)
    np.testing.assert_array_equal(fe[:, emb.solid == 1], g0[:, emb.solid == 1])


@pytest.mark.parametrize("tau,steps", [(2.0, 2000), (1.0, 6000)])
def test_body_force_poiseuille_is_exact(orc, tau, steps):
    # eq. gravity drives the flow; at steady state the velocity after the boundary
    # rule (stored velocity minus F / rho, reading R11) is the parabola of
    # eq. poiseuille with the viscosity of eq. visc, zero on the wall nodes
    wl = inp.force_poiseuille(n=16, tau=tau, force=1e-5, wall_axis=0, flow_axis=2, other=3)
    lat = orc.Lattice.from_workload(wl)
    f = orc.run(lat, orc.init_equilibrium(lat), steps)
    rho, u = orc.macros(lat, f)
    F = wl.force[2]
    u_pre = u[2] - F / rho
    x = np.arange(wl.nx)
    h = (wl.nx - 1) / 2.0
    eta = rho * (tau - 0.5) / 3.0
    exact = F / (2.0 * eta) * (h * h - (x - h) ** 2)
    assert np.abs(u_pre - exact).max() < 1e-10 * exact.max()
    assert np.abs(u_pre[:, :, [0, -1]]).max() < 1e-16
    assert np.abs(u[:2]).max() < 1e-15


def mirror(orc, f, axis):
    c, _, _ = orc.lattice()
    index = {tuple(v): k for k, v in enumerate(c)}
    flip = np.ones(3, int)
    flip[axis] = -1
    perm = np.array([index[tuple(flip * c[k])] for k in range(19)])
    out = np.empty_like(f)
    out[perm] = np.flip(f, axis=3 - axis)
    return out


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_pillar_flow_is_mirror_symmetric(orc, axis):
    flow = [a for a in range(3) if a != axis][0]
    side = [a for a in range(3) if a not in (axis, flow)][0]
    wl = inp.pillar_channel(axis=axis, flow=flow)
    lat = orc.Lattice.from_workload(wl)
    f = orc.run(lat, orc.init_equilibrium(lat), 60)
    assert np.abs(f - orc.init_equilibrium(lat)).max() > 1e-7       # the force set it moving
    for ax in (axis, side):
        np.testing.assert_allclose(mirror(orc, f, ax), f, rtol=0, atol=1e-14, err_msg=f"mirror {ax}")


@pytest.mark.parametrize("axis", [0, 2])
def test_pillar_boundary_nodes_hold_the_prescribed_momenta(orc, axis):
    # After the boundary rule a no-slip plane, concave edge or corner node has zero
    # momentum, a convex edge none along the edge, a junction none through its plane;
    # the collision then adds F (eq. gravity), so the stored momentum shows F there.
    flow = [a for a in range(3) if a != axis][0]
    wl = inp.pillar_channel(axis=axis, flow=flow)
    lat = orc.Lattice.from_workload(wl)
    f = orc.run(lat, orc.init_equilibrium(lat), 40)
    c, _, _ = orc.lattice()
    j = np.einsum("kzyx,ka->azyx", f, c.astype(float))
    F = wl.force
    e = np.zeros(3)
    e[axis] = 1.0
    code = wl.code
    full = (code >= 1) & (code <= 18)
    assert full.any()
    np.testing.assert_allclose(j[:, full].T, np.broadcast_to(F, (full.sum(), 3)), rtol=0, atol=5e-16)
    convex = code < 0
    assert convex.any()
    assert np.abs(np.einsum("a,an->n", e, j[:, convex])).max() < 5e-16
    junction = code >= 27
    assert junction.any()
    assert np.abs(np.einsum("a,an->n", e, j[:, junction])).max() < 5e-16


def test_inconsistent_codes_are_rejected(orc):
    wl = inp.pillar_channel()
    node = tuple(np.argwhere(wl.code == -12)[0])
    wl.code[node] = -7                      # a convex edge facing the wrong way
    lat = orc.Lattice.from_workload(wl)
    nz, ny, nx = wl.code.shape
    assert orc.check_geometry(lat) == (node[0] * ny + node[1]) * nx + node[2]
    with pytest.raises(RuntimeError):
        orc.step(lat, orc.init_equilibrium(lat))
    wl2 = inp.pillar_channel()
    wl2.code[0, 0, 0] = 51                  # not a code
    with pytest.raises(RuntimeError):
        orc.step(orc.Lattice.from_workload(wl2), orc.init_equilibrium(orc.Lattice.from_workload(wl2)))
