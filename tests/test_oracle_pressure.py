"""Pins of the oracle's pressure (density) variant, CPU only.

The paper gives, for every plane, the normal velocity that a prescribed density rho0
implies (eq. rhoin and the appendix), keeps the unknown-population rules of the
velocity closure, and fixes the edge and corner densities next to a pressure plane
(eq. buried_rho, corner variant). Pins: the printed relations (golden fixture), the
exact density and tangential velocity after the closure, a least-squares solve of the
ansatz with the normal velocity as unknown, equilibrium reproduction, agreement of the
explicit and compact forms, lattice symmetry, and the paper's second-order convergence
of the pressure-driven square duct against its analytic series.
"""
import itertools
import json
import os

import numpy as np
import pytest

import lbm_inputs as inp

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "d3q19_paper_sets.json")))
FACES = range(6)


def normal(face):
    n = np.zeros(3, int)
    n[face // 2] = 1 if face % 2 == 0 else -1
    return n


def face_of(n):
    a = int(np.argmax(np.abs(n)))
    return 2 * a + (0 if n[a] > 0 else 1)


def unknown_set(c, normals):
    return [k for k in range(19) if any(c[k] @ n > 0 for n in normals)]


def random_state(orc, seed, rho=1.0, u=(0.02, -0.01, 0.015), amp=0.2):
    return orc.feq(rho, u) * (1 + amp * inp.noise(seed, (19,)))


def signed_perms():
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            P = np.zeros((3, 3), int)
            for i in range(3):
                P[i, perm[i]] = signs[i]
            yield P


def pop_map(c, P):
    idx = {tuple(v): k for k, v in enumerate(c)}
    return np.array([idx[tuple(P @ c[k])] for k in range(19)])


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("face", FACES)
@pytest.mark.parametrize("seed", range(4))
def test_density_and_tangential_velocity_are_exact(orc, face, form, seed):
    r = inp.uniform(seed, 21, np.arange(4))
    rho0 = 0.97 + 0.06 * r[0]
    ut = 0.08 * (2 * r[1:] - 1)
    f = random_state(orc, 100 + seed)
    g, vn = orc.close_face_pressure(face, f, rho0, ut, form)
    rho, u = orc.moments(g)
    assert abs(rho - rho0) < 1e-15
    a = face // 2
    for b in range(3):
        if b != a:
            assert abs(u[b] - ut[b]) < 1e-15
    assert abs(u[a] - vn) < 1e-15
    # the normal velocity is the printed relation applied to the known populations
    rel = GOLD["density_relations"][str(face)]
    S = sum(f[i - 1] for i in rel["once"]) + 2 * sum(f[i - 1] for i in rel["twice"])
    form_txt = GOLD["pressure_variant"]["normal_velocity"][str(face)]["form"]
    want = 1 - S / rho0 if form_txt.startswith("1") else -1 + S / rho0
    assert abs(vn - want) < 1e-15


@pytest.mark.parametrize("face", FACES)
@pytest.mark.parametrize("seed", range(3))
def test_pressure_closure_equals_least_squares_solution(orc, face, seed):
    # Unknowns: the five incoming f_i, the normal velocity u_n, N_t1, N_t2. Equations:
    # density = rho0, momentum = rho0 (u_t + u_n n), and the non-equilibrium bounce-back
    # ansatz f_i - f_-i = f_i^eq - f_-i^eq - t_i.N, linear in u_n at fixed rho0.
    c, _, opp = orc.lattice()
    n = normal(face)
    a = face // 2
    unk = unknown_set(c, [n])
    known = [k for k in range(19) if k not in unk]
    tang = [b for b in range(3) if b != a]
    r = inp.uniform(seed, 23, np.arange(4))
    rho0 = 0.98 + 0.04 * r[0]
    ut = 0.06 * (2 * r[1:] - 1)
    ut[a] = 0.0
    f = random_state(orc, 200 + seed)
    # f^eq_i(rho, u) - f^eq_-i(rho, u) is rho times a linear form in u whose coefficient
    # along axis b is f^eq_i(1, e_b) - f^eq_i(1, -e_b) (the oracle's own, separately
    # pinned equilibrium; c_-i = -c_i turns the pair difference into the sign flip)
    d_axis = [orc.feq(1.0, np.eye(3)[b]) - orc.feq(1.0, -np.eye(3)[b]) for b in range(3)]
    nu = len(unk)
    A = np.zeros((4 + nu, nu + 3))
    bvec = np.zeros(4 + nu)
    for j, k in enumerate(unk):
        A[0, j] = 1.0
        A[1:4, j] = c[k]
    A[1 + a, nu] = -rho0                  # x[nu] = v_a, the velocity along the axis
    bvec[0] = rho0 - f[known].sum()
    bvec[1:4] = rho0 * ut - f[known] @ c[known]
    for r_, k in enumerate(unk):
        row = 4 + r_
        A[row, r_] = 1.0
        A[row, nu] = -rho0 * d_axis[a][k]
        t = c[k] - (c[k] @ n) * n
        for m, b in enumerate(tang):
            A[row, nu + 1 + m] = t[b]
        bvec[row] = f[opp[k]] + rho0 * sum(ut[b] * d_axis[b][k] for b in tang)
    x, _, rank, _ = np.linalg.lstsq(A, bvec, rcond=None)
    assert rank == nu + 3
    np.testing.assert_allclose(A @ x, bvec, atol=1e-14)
    for form in (0, 1):
        g, vn = orc.close_face_pressure(face, f, rho0, ut, form)
        np.testing.assert_allclose(g[unk], x[:nu], rtol=0, atol=1e-14)
        assert abs(vn - x[nu]) < 1e-14


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("face", FACES)
def test_pressure_closure_reproduces_equilibrium(orc, face, form):
    c, _, _ = orc.lattice()
    rho0, u = 1.013, np.array([0.021, -0.017, 0.032])
    feq = orc.feq(rho0, u)
    f = feq.copy()
    f[unknown_set(c, [normal(face)])] = 7.0
    g, vn = orc.close_face_pressure(face, f, rho0, u, form)
    np.testing.assert_allclose(g, feq, rtol=0, atol=1e-15)
    assert abs(vn - u[face // 2]) < 1e-15


def test_pressure_faces_are_symmetry_images(orc):
    c, _, _ = orc.lattice()
    ut = np.array([0.031, -0.017, 0.023])
    f = random_state(orc, 41)
    for face in FACES:
        u = ut.copy()
        u[face // 2] = 0.0
        g, vn = orc.close_face_pressure(face, f, 1.01, u, 0)
        for P in signed_perms():
            pi = pop_map(c, P)
            fi = np.empty(19)
            fi[pi] = f
            img = face_of(P @ normal(face))
            gi, vni = orc.close_face_pressure(img, fi, 1.01, P @ u, 0)
            np.testing.assert_allclose(gi[pi], g, rtol=0, atol=1e-15)


EDGES = [(a, b) for a in FACES for b in FACES if a // 2 < b // 2]
CORNERS = [(x, y, z) for x in (0, 1) for y in (2, 3) for z in (4, 5)]


@pytest.mark.parametrize("edge", EDGES)
def test_pressure_edge_density_and_no_slip(orc, edge):
    c, _, _ = orc.lattice()
    n1, n2 = normal(edge[0]), normal(edge[1])
    f = random_state(orc, 300 + 6 * edge[0] + edge[1])
    g = orc.close_edge(*edge, f, rho_p=1.023)
    rho, u = orc.moments(g)
    assert abs(rho - 1.023) < 1e-15
    np.testing.assert_allclose(u, 0, atol=1e-16)
    buried = [k for k in range(18) if (c[k] == n1 - n2).all() or (c[k] == n2 - n1).all()]
    plain = orc.close_edge(*edge, f)
    fb = plain[buried[0]]  # the velocity rule's buried value = (sum of 16) / 22
    eb = GOLD["pressure_variant"]["edge_buried"]
    want = (1.023 - eb["numerator_factor"] * fb) / eb["divisor"]
    assert abs(g[buried[0]] - want) < 1e-15 and abs(g[buried[1]] - want) < 1e-15
    assert abs(g[18] - eb["rest_factor"] * want) < 1e-15
    moving = [k for k in range(18) if k not in buried]
    np.testing.assert_array_equal(g[moving], plain[moving])


@pytest.mark.parametrize("corner", CORNERS)
def test_pressure_corner_density_and_no_slip(orc, corner):
    c, _, _ = orc.lattice()
    f = random_state(orc, 400 + corner[0] + 2 * corner[1])
    g = orc.close_corner(*corner, f, rho_p=0.987)
    rho, u = orc.moments(g)
    assert abs(rho - 0.987) < 1e-15
    np.testing.assert_allclose(u, 0, atol=1e-16)
    s = sum(normal(x) for x in corner)
    buried = [k for k in range(18) if c[k] @ s == 0]
    plain = orc.close_corner(*corner, f)
    cb = GOLD["pressure_variant"]["corner_buried"]
    want = 0.987 / cb["rho_divisor"] - plain[buried[0]]
    for k in buried:
        assert abs(g[k] - want) < 1e-15
    assert abs(g[18] - cb["rest_factor"] * want) < 1e-15


def test_pressure_planes_hold_their_density_every_step(orc):
    wl = inp.pressure_duct(7, 11, 0.8, 1.004, 0.996)
    lat = orc.Lattice.from_workload(wl)
    f = orc.init_equilibrium(lat) * (1 + 0.01 * inp.noise(5, lat.shape))
    for _ in range(5):
        f = orc.step(lat, f)
        rho, u = orc.macros(lat, f)
        np.testing.assert_allclose(rho[:, :, 0], 1.004, rtol=0, atol=2e-15)    # faces, edges, corners
        np.testing.assert_allclose(rho[:, :, -1], 0.996, rtol=0, atol=2e-15)
        np.testing.assert_allclose(u[1:, 1:-1, 1:-1, 0], 0, atol=2e-16)          # no tangential velocity
        np.testing.assert_allclose(u[:, [0, -1], :, :], 0, atol=2e-16)           # walls (incl. edges)


def test_lattice_rejects_two_pressure_axes(orc):
    wl = inp.make_workload("bad", 6, 6, 6, 1.0, [None] * 4 + [inp.ZERO, inp.ZERO],
                           face_p=[1.0, 1.0, 1.0, 1.0, None, None])
    lat = orc.Lattice.from_workload(wl)
    with pytest.raises(RuntimeError):
        orc.step(lat, orc.init_equilibrium(lat))


def square_duct_series(n, terms=50):
    b = n - 1.0
    s = np.arange(n) - (n - 1) / 2.0
    X, Y = np.meshgrid(s, s, indexing="ij")
    C = np.zeros_like(X)
    for m in range(terms):
        k = 2 * m + 1
        C += (-1) ** m * np.cosh(k * np.pi * X / b) * np.cos(k * np.pi * Y / b) / (k ** 3 * np.cosh(k * np.pi / 2))
    return b * b / 4 - Y ** 2 - C * 8 * b * b / np.pi ** 3


@pytest.mark.slow
def test_pressure_driven_square_duct_converges_at_second_order(orc):
    # The paper's square-channel test: pressure planes at both ends, no-slip walls,
    # edges and corners; the velocity in a cross-section against eq. squarechannel
    # with the local pressure gradient and eta = c_s^2 rho (tau - 1/2) (eq. visc).
    errs, widths = [], []
    for n in (9, 13, 17):
        length = 3 * n
        wl = inp.pressure_duct(n, length, 1.0, 1.002, 0.998)
        lat = orc.Lattice.from_workload(wl)
        f = orc.run(lat, orc.init_equilibrium(lat), 14 * n * n)
        rho, u = orc.macros(lat, f)
        xm = length // 2
        grad = (rho[:, :, xm + 1].mean() - rho[:, :, xm - 1].mean()) / 2.0 / 3.0
        eta = rho[:, :, xm].mean() * (1.0 - 0.5) / 3.0
        an = -grad / (2 * eta) * square_duct_series(n)
        errs.append(np.sqrt(((u[0][:, :, xm] - an) ** 2).mean() / (an ** 2).mean()))
        widths.append(n - 1)
    slopes = [np.log(errs[i] / errs[i + 1]) / np.log(widths[i + 1] / widths[i]) for i in range(2)]
    target = GOLD["pressure_variant"]["duct_error_slope"]["value"]
    for s in slopes:
        assert abs(s - target) < 0.3, slopes
