"""Pins of the oracle's boundary closures (face, edge, corner), CPU only.

Each property is fixed by the paper or by mathematics:
  * the printed density relations and unknown sets (golden fixture);
  * equilibrium states are reproduced exactly (the N corrections vanish there);
  * the velocity on a closed node is exactly the prescribed one;
  * a LAPACK least-squares solve of the paper's ansatz (non-equilibrium bounce-back
    with two transverse corrections) plus the moment equations gives the same
    unknowns and density;
  * the explicit per-plane formulas and the compact rule agree;
  * all faces, edges and corners are images of each other under the lattice's
    rotations and reflections;
  * edges and corners carry zero momentum and a rest/buried split fixed by the
    lattice weights.
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
    base = orc.feq(rho, u)
    return base * (1 + amp * inp.noise(seed, (19,)))


def signed_perms():
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            P = np.zeros((3, 3), int)
            for i in range(3):
                P[i, perm[i]] = signs[i]
            yield P


def pop_map(c, P):
    """pi with c[pi[k]] = P c[k]."""
    idx = {tuple(v): k for k, v in enumerate(c)}
    return np.array([idx[tuple(P @ c[k])] for k in range(19)])


# ---------------------------------------------------------------------------------
# faces
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("face", FACES)
def test_unknown_sets_match_paper(orc, face):
    c, _, _ = orc.lattice()
    got = [k + 1 for k in unknown_set(c, [normal(face)])]
    assert sorted(got) == sorted(GOLD["unknown_after_streaming"][str(face)])


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("face", FACES)
def test_density_relation_matches_paper(orc, face, form):
    # Probe the closure's rho with unit populations: rho(e_k) * (1 - u.n) must be 1 for
    # the printed "once" set, 2 for the "twice" set and 0 for the unknown ones.
    g = GOLD["density_relations"][str(face)]
    u = np.array([0.03, -0.02, 0.01])
    n = normal(face)
    for k in range(19):
        f = np.zeros(19)
        f[k] = 1.0
        _, rho = orc.close_face(face, f, u, form)
        coef = rho * (1 - u @ n)
        expect = 1.0 if (k + 1) in g["once"] else (2.0 if (k + 1) in g["twice"] else 0.0)
        assert abs(coef - expect) < 1e-15, (face, k + 1)
    sign = g["denominator"].split()[1]
    assert (sign == "-") == (n[face // 2] > 0)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("face", FACES)
@pytest.mark.parametrize("seed", range(4))
def test_equilibrium_is_reproduced(orc, face, form, seed):
    # N^z_x and N^z_y vanish at equilibrium, so the closure returns f_eq exactly
    # whatever the unknown populations held before.
    c, _, _ = orc.lattice()
    r = inp.uniform(seed, 7, np.arange(4))
    rho = 0.9 + 0.2 * r[0]
    u = 0.08 * (2 * r[1:] - 1)
    feq = orc.feq(rho, u)
    f = feq.copy()
    for k in unknown_set(c, [normal(face)]):
        f[k] = 123.0 + k
    g, rho_c = orc.close_face(face, f, u, form)
    np.testing.assert_allclose(g, feq, rtol=0, atol=2e-16)
    assert abs(rho_c - rho) < 1e-15


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("face", FACES)
@pytest.mark.parametrize("seed", range(6))
def test_prescribed_velocity_is_exact(orc, face, form, seed):
    # After the closure the node's moments give exactly the prescribed velocity and
    # the density the closure reports.
    r = inp.uniform(seed, 9, np.arange(3))
    u = 0.1 * (2 * r - 1)
    f = random_state(orc, seed + 10)
    g, rho_c = orc.close_face(face, f, u, form)
    rho, v = orc.moments(g)
    assert abs(rho - rho_c) < 1e-14
    np.testing.assert_allclose(v, u, rtol=0, atol=1e-15)


@pytest.mark.parametrize("face", FACES)
@pytest.mark.parametrize("seed", range(6))
def test_explicit_and_compact_forms_agree(orc, face, seed):
    u = 0.1 * (2 * inp.uniform(seed, 11, np.arange(3)) - 1)
    f = random_state(orc, seed + 20)
    g0, r0 = orc.close_face(face, f, u, 0)
    g1, r1 = orc.close_face(face, f, u, 1)
    np.testing.assert_allclose(g0, g1, rtol=0, atol=1e-15)
    assert abs(r0 - r1) < 1e-15


@pytest.mark.parametrize("face", FACES)
@pytest.mark.parametrize("seed", range(4))
def test_closure_equals_least_squares_solution(orc, face, seed):
    # Unknowns x = (the five f_i pointing in, rho, N_t1, N_t2). Equations: density and
    # the three velocity components (eqs. rho, vel) plus, for every unknown i, the
    # bounce-back of the non-equilibrium part corrected by the transverse momentum
    #   f_i - f_-i = f_i^eq(rho, u) - f_-i^eq(rho, u) - t_i . N,
    # 9 equations, rank 8. f^eq is linear in rho at fixed u, so the system is linear.
    c, _, opp = orc.lattice()
    n = normal(face)
    unk = unknown_set(c, [n])
    known = [k for k in range(19) if k not in unk]
    tang = [a for a in range(3) if n[a] == 0]
    u = 0.1 * (2 * inp.uniform(seed, 13, np.arange(3)) - 1)
    f = random_state(orc, seed + 30)
    d_eq = orc.feq(1.0, u)  # per unit density
    A = np.zeros((4 + len(unk), len(unk) + 3))
    b = np.zeros(4 + len(unk))
    for j, k in enumerate(unk):
        A[0, j] = 1.0
        A[1:4, j] = c[k]
    A[0, len(unk)] = -1.0
    A[1:4, len(unk)] = -u
    b[0] = -f[known].sum()
    b[1:4] = -(f[known] @ c[known])
    for r, k in enumerate(unk):
        row = 4 + r
        A[row, r] = 1.0
        A[row, len(unk)] = -(d_eq[k] - d_eq[opp[k]])
        t = c[k] - (c[k] @ n) * n
        for m, a in enumerate(tang):
            A[row, len(unk) + 1 + m] = t[a]
        b[row] = f[opp[k]]
    x, res, rank, _ = np.linalg.lstsq(A, b, rcond=None)
    assert rank == len(unk) + 3
    np.testing.assert_allclose(A @ x, b, atol=1e-14)  # consistent system
    for form in (0, 1):
        g, rho = orc.close_face(face, f, u, form)
        np.testing.assert_allclose(g[unk], x[:len(unk)], rtol=0, atol=1e-14)
        assert abs(rho - x[len(unk)]) < 1e-14


@pytest.mark.parametrize("form", [0, 1])
def test_faces_are_symmetry_images(orc, form):
    # For every signed permutation P of the axes, closing the image state on the
    # image face with the image velocity gives the image of the closed state. This
    # ties all six per-plane formula sets to each other.
    c, _, _ = orc.lattice()
    u = np.array([0.031, -0.017, 0.023])
    f = random_state(orc, 41)
    for face in FACES:
        g, rho = orc.close_face(face, f, u, form)
        for P in signed_perms():
            pi = pop_map(c, P)
            fi = np.empty(19)
            fi[pi] = f
            gi, rhoi = orc.close_face(face_of(P @ normal(face)), fi, P @ u, form)
            np.testing.assert_allclose(gi[pi], g, rtol=0, atol=1e-15)
            assert abs(rhoi - rho) < 1e-15


# ---------------------------------------------------------------------------------
# edges
# ---------------------------------------------------------------------------------

EDGES = [(a, b) for a in FACES for b in FACES if a // 2 < b // 2]
CORNERS = [(x, y, z) for x in (0, 1) for y in (2, 3) for z in (4, 5)]


@pytest.mark.parametrize("edge", EDGES)
def test_edge_zero_momentum_and_weights(orc, edge):
    # eq. edge / eq. buried: no-slip on the node, buried links equal, rest population
    # twelve times a buried link, density 36 times a buried link.
    c, _, _ = orc.lattice()
    n1, n2 = normal(edge[0]), normal(edge[1])
    f = random_state(orc, 50 + edge[0] * 6 + edge[1])
    g = orc.close_edge(*edge, f)
    rho, v = orc.moments(g)
    np.testing.assert_allclose(v, 0, atol=1e-16)
    buried = [k for k in range(18) if (c[k] == n1 - n2).all() or (c[k] == n2 - n1).all()]
    assert len(buried) == 2
    fb = g[buried[0]]
    assert g[buried[1]] == fb
    assert abs(g[18] - 12 * fb) < 1e-15
    assert abs(rho - 36 * fb) < 1e-15
    bw = GOLD["buried_weights"]["edge"]
    moving = [k for k in range(18) if k not in buried]
    assert sum(1 for k in moving if k < 6) == bw["axis_terms"]
    assert sum(1 for k in moving if k >= 6) == bw["diagonal_terms"]
    assert abs(fb - g[moving].sum() / bw["divisor"]) < 1e-16


@pytest.mark.parametrize("edge", EDGES)
def test_edge_reproduces_rest_equilibrium(orc, edge):
    c, _, _ = orc.lattice()
    feq = orc.feq(1.07, [0, 0, 0])
    f = feq.copy()
    for k in unknown_set(c, [normal(edge[0]), normal(edge[1])]):
        f[k] = -5.0
    np.testing.assert_allclose(orc.close_edge(*edge, f), feq, rtol=0, atol=1e-15)


def test_edge_matches_printed_example(orc):
    # The y-directed edge between z=0 and x=0: after bounce-back the remaining y
    # momentum is f3 - f4, removed in quarters from f7, f8, f15, f17.
    ex = GOLD["edge_example"]
    c, _, opp = orc.lattice()
    f = random_state(orc, 60)
    g = orc.close_edge(*ex["faces"], f)
    d = ex["correction_prefactor"] * (f[2] - f[3])
    for i in ex["corrected"]:
        k = i - 1
        assert abs(g[k] - (f[opp[k]] - c[k, 1] * d)) < 1e-16, i
    unk = unknown_set(c, [normal(ex["faces"][0]), normal(ex["faces"][1])])
    for k in range(19):
        if k not in unk and k != 18:
            assert g[k] == f[k]
    bounced_plain = sorted(set(k + 1 for k in unk) - {10, 13} - set(ex["corrected"]))
    for i in bounced_plain:
        assert g[i - 1] == f[opp[i - 1]]


def test_edges_are_symmetry_images(orc):
    c, _, _ = orc.lattice()
    f = random_state(orc, 61)
    for e in EDGES:
        g = orc.close_edge(*e, f)
        for P in signed_perms():
            pi = pop_map(c, P)
            fi = np.empty(19)
            fi[pi] = f
            fa, fb = face_of(P @ normal(e[0])), face_of(P @ normal(e[1]))
            if fa // 2 > fb // 2:
                fa, fb = fb, fa
            gi = orc.close_edge(fa, fb, fi)
            np.testing.assert_allclose(gi[pi], g, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------------
# corners
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("corner", CORNERS)
def test_corner_zero_momentum_and_weights(orc, corner):
    c, _, _ = orc.lattice()
    s = sum(normal(fc) for fc in corner)
    f = random_state(orc, 70 + corner[0] + 2 * corner[1] + 4 * corner[2])
    g = orc.close_corner(*corner, f)
    rho, v = orc.moments(g)
    np.testing.assert_allclose(v, 0, atol=1e-16)
    buried = [k for k in range(18) if c[k] @ s == 0]
    bw = GOLD["buried_weights"]["corner"]
    assert len(buried) == bw["buried"]
    fb = g[buried[0]]
    assert all(g[k] == fb for k in buried)
    assert abs(g[18] - bw["rest_factor"] * fb) < 1e-15
    assert abs(rho - 36 * fb) < 1e-15
    moving = [k for k in range(18) if k not in buried]
    assert abs(fb - g[moving].sum() / bw["divisor"]) < 1e-16


@pytest.mark.parametrize("corner", CORNERS)
def test_corner_reproduces_rest_equilibrium(orc, corner):
    c, _, _ = orc.lattice()
    feq = orc.feq(0.96, [0, 0, 0])
    f = feq.copy()
    for k in unknown_set(c, [normal(fc) for fc in corner]):
        f[k] = 9.0
    np.testing.assert_allclose(orc.close_corner(*corner, f), feq, rtol=0, atol=1e-15)


def test_corners_are_symmetry_images(orc):
    c, _, _ = orc.lattice()
    f = random_state(orc, 71)
    for cr in CORNERS:
        g = orc.close_corner(*cr, f)
        for P in signed_perms():
            pi = pop_map(c, P)
            fi = np.empty(19)
            fi[pi] = f
            img = sorted(face_of(P @ normal(fc)) for fc in cr)
            gi = orc.close_corner(*img, fi)
            np.testing.assert_allclose(gi[pi], g, rtol=0, atol=1e-15)


def test_closure_ignores_unknown_inputs(orc):
    # Only populations known after streaming may enter a closure.
    c, _, _ = orc.lattice()
    f = random_state(orc, 80)
    u = [0.01, 0.02, -0.03]
    for face in FACES:
        unk = unknown_set(c, [normal(face)])
        h = f.copy()
        h[unk] = np.nan
        for form in (0, 1):
            g, _ = orc.close_face(face, h, u, form)
            assert np.isfinite(g).all()
    for e in EDGES:
        h = f.copy()
        h[unknown_set(c, [normal(e[0]), normal(e[1])])] = np.nan
        assert np.isfinite(orc.close_edge(*e, h)).all()
    for cr in CORNERS:
        h = f.copy()
        h[unknown_set(c, [normal(x) for x in cr])] = np.nan
        assert np.isfinite(orc.close_corner(*cr, h)).all()
