"""Pins of the oracle's reductions (CPU only): mass, |u - u_prev|^2, |u|^2 and the
bad-node count of ``orc_reduce`` against an independent numpy computation.

The velocity set used here is built from the paper's printed component sets (eqs. vx,
vy, vz, stored in tests/golden/), not from the oracle's tables, and density and
velocity follow their definitions (eq. rho, eq. vel) written as array operations, so a
wrong sign, index or layout in the oracle's per-node loop fails one of these checks.
The bad-node rule -- a node whose density is not finite or not positive, or whose
velocity is not finite -- is the failure criterion of the residual check; the paper
has no counterpart.
"""
import json
import os

import numpy as np
import pytest

import lbm_inputs as inp

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "d3q19_paper_sets.json")))


def paper_velocities():
    """c[19, 3] from the printed sets: population i has c_a = +1 if listed under
    'plus' for axis a, -1 under 'minus', else 0 (population 19 is the rest vector)."""
    c = np.zeros((19, 3))
    for a, name in enumerate("xyz"):
        for i in GOLD["velocity_components"][name]["plus"]:
            c[i - 1, a] = 1
        for i in GOLD["velocity_components"][name]["minus"]:
            c[i - 1, a] = -1
    return c


def numpy_reduce(f, u_prev):
    """The four sums from the definitions, as whole-array numpy operations."""
    c = paper_velocities()
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        rho = f.sum(axis=0)
        u = np.einsum("ka,kzyx->azyx", c, f) / rho
        up = np.zeros_like(u) if u_prev is None else u_prev
        du2 = ((u - up) ** 2).sum()
        u2 = (u ** 2).sum()
        bad = ~np.isfinite(rho) | ~(rho > 0) | ~np.isfinite(u).all(axis=0)
    return np.array([rho.sum(), du2, u2, float(bad.sum())]), u


def state(seed, shape, u=(0.02, -0.01, 0.015), amp=0.05):
    """f = f_eq(1, u) (1 + amp eps): the equilibrium written out from eq. feq with the
    paper's weights, not taken from the oracle."""
    c = paper_velocities()
    num = GOLD["weights"]["numerators_over_36"]
    w = np.array([num["1-6"]] * 6 + [num["7-18"]] * 12 + [num["19"]]) / 36.0
    cu = c @ np.asarray(u)
    feq = w * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * np.dot(u, u))
    return feq[:, None, None, None] * (1 + amp * inp.noise(seed, shape))


DIMS = [(7, 5, 3), (13, 4, 6), (1, 1, 1)]


@pytest.mark.parametrize("dims", DIMS)
def test_reduce_matches_definitions(orc, dims):
    nx, ny, nz = dims
    lat = orc.Lattice(nx, ny, nz, [0] * 6, [None] * 6, 1.0)
    f = state(3, lat.shape)
    # a previous velocity field with a different value on every node and component, so
    # that a transposed or shifted index in the oracle changes the sum
    u_prev = 0.01 * (2 * inp.uniform(9, 1, np.arange(3 * nx * ny * nz)) - 1).reshape(3, nz, ny, nx)
    got = orc.reduce(lat, f, u_prev)
    ref, u = numpy_reduce(f, u_prev)
    np.testing.assert_allclose(got[:3], ref[:3], rtol=1e-13, atol=0)
    assert got[3] == 0 == ref[3]
    # the oracle's macroscopic routine gives the same velocities the sums were formed of
    _, uo = orc.macros(lat, f)
    np.testing.assert_allclose(uo, u, rtol=0, atol=1e-16)


def test_reduce_without_previous_velocity_takes_zero(orc):
    lat = orc.Lattice(6, 5, 4, [0] * 6, [None] * 6, 1.0)
    f = state(4, lat.shape)
    got = orc.reduce(lat, f, None)
    ref, _ = numpy_reduce(f, None)
    np.testing.assert_allclose(got[:3], ref[:3], rtol=1e-13, atol=0)
    assert got[1] == got[2]
    # residual as the ratio of the two sums; with u_prev = u it is exactly zero
    _, u = orc.macros(lat, f)
    assert orc.residual(lat, f, None) == pytest.approx(1.0, abs=1e-15)
    assert orc.residual(lat, f, u) == 0.0


def test_mass_is_the_sum_of_all_populations(orc):
    # mass = sum over nodes and populations, in any order, to rounding
    lat = orc.Lattice(9, 7, 5, [0] * 6, [None] * 6, 1.0)
    f = state(5, lat.shape)
    got = orc.reduce(lat, f, None)
    assert got[0] == pytest.approx(float(np.sum(f, dtype=np.float64)), rel=1e-14)


@pytest.mark.parametrize("kind", ["negative", "zero", "nan", "inf", "nan_velocity_only"])
def test_bad_node_count(orc, kind):
    nx, ny, nz = 8, 5, 4
    lat = orc.Lattice(nx, ny, nz, [0] * 6, [None] * 6, 1.0)
    f = state(6, lat.shape)
    bad_nodes = [(1, 2, 3), (3, 0, 6)]            # (z, y, x)
    for z, y, x in bad_nodes:
        if kind == "negative":
            f[:, z, y, x] *= -1.0                  # density < 0, velocity finite
        elif kind == "zero":
            f[:, z, y, x] = 0.0                    # density 0: velocity 0/0
        elif kind == "nan":
            f[4, z, y, x] = np.nan
        elif kind == "inf":
            f[0, z, y, x] = np.inf
        else:
            # populations 1 (c_x = +1) and 2 (c_x = -1) of opposite sign: they cancel in
            # the density, which stays finite and positive, but the x momentum
            # 1e308 - (-1e308) overflows, so only the velocity check flags the node
            f[0, z, y, x] = 1e308
            f[1, z, y, x] = -1e308
    got = orc.reduce(lat, f, None)
    ref, _ = numpy_reduce(f, None)
    assert got[3] == ref[3] == len(bad_nodes), (got, ref)
    if kind == "negative":
        # every sum stays finite and still follows the definitions
        np.testing.assert_allclose(got[:3], ref[:3], rtol=1e-13, atol=0)
    else:
        assert not np.isfinite(got[:3]).all()


def test_bad_node_count_distinguishes_nodes(orc):
    # the count is per node, not per population: three bad populations on one node
    # count once, one bad population on each of two nodes counts twice
    lat = orc.Lattice(5, 4, 3, [0] * 6, [None] * 6, 1.0)
    f = state(7, lat.shape)
    f[[0, 5, 9], 1, 1, 1] = np.nan
    assert orc.reduce(lat, f, None)[3] == 1
    f[2, 2, 3, 4] = np.nan
    assert orc.reduce(lat, f, None)[3] == 2
