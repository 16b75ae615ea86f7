"""Pins of the oracle's lattice tables, equilibrium and collision (CPU only).

Every expectation here comes from the paper's printed index sets or from closed-form
properties of the D3Q19 lattice, never from the oracle itself.
"""
import json
import os

import numpy as np
import pytest

import lbm_inputs as inp

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "d3q19_paper_sets.json")))


def test_velocity_set_matches_printed_component_sums(orc):
    # eqs. vx, vy, vz list, for each axis, the populations with c = +1 and c = -1.
    c, _, _ = orc.lattice()
    for a, name in enumerate("xyz"):
        plus = sorted(k + 1 for k in range(19) if c[k, a] == 1)
        minus = sorted(k + 1 for k in range(19) if c[k, a] == -1)
        assert plus == sorted(GOLD["velocity_components"][name]["plus"])
        assert minus == sorted(GOLD["velocity_components"][name]["minus"])
    assert (c[18] == 0).all()
    assert len({tuple(v) for v in c}) == 19


def test_weights_and_isotropy(orc):
    c, w, opp = orc.lattice()
    num = GOLD["weights"]["numerators_over_36"]
    np.testing.assert_array_equal(w * 36, [num["1-6"]] * 6 + [num["7-18"]] * 12 + [num["19"]])
    assert abs(w.sum() - 1) < 1e-15
    # c_s^2 = 1/3 and the fourth-order isotropy that the second-order equilibrium needs
    m2 = np.einsum("k,ka,kb->ab", w, c, c)
    np.testing.assert_allclose(m2, np.eye(3) / 3, atol=1e-15)
    np.testing.assert_allclose(np.einsum("k,ka->a", w, c), 0, atol=1e-15)
    m4 = np.einsum("k,ka,kb,kc,kd->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    np.testing.assert_allclose(m4, iso, atol=1e-15)
    for k in range(19):
        np.testing.assert_array_equal(c[opp[k]], -c[k])


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(orc, seed):
    # eq. feq: zeroth, first and second moments have closed forms.
    r = inp.uniform(seed, 0, np.arange(4))
    rho = 0.8 + 0.4 * r[0]
    u = 0.1 * (2 * r[1:] - 1)
    c, _, _ = orc.lattice()
    f = orc.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-15
    np.testing.assert_allclose(f @ c, rho * u, atol=1e-16)
    pi = np.einsum("k,ka,kb->ab", f, c, c)
    np.testing.assert_allclose(pi, rho * np.eye(3) / 3 + rho * np.outer(u, u), atol=1e-15)
    m, v = orc.moments(f)
    assert abs(m - rho) < 1e-15
    np.testing.assert_allclose(v, u, atol=1e-16)


@pytest.mark.parametrize("tau", [0.55, 1.0, 1.7])
def test_bgk_collision(orc, tau):
    # eq. bgk: density and velocity are invariants; the non-equilibrium part scales
    # by (1 - 1/tau).
    base = orc.feq(1.02, [0.03, -0.01, 0.02])
    f = base * (1 + 0.05 * inp.noise(3, (19,)))
    rho, u = orc.moments(f)
    g = orc.collide(f, tau)
    rho2, u2 = orc.moments(g)
    assert abs(rho2 - rho) < 1e-15
    np.testing.assert_allclose(u2, u, atol=1e-16)
    feq = orc.feq(rho, u)
    np.testing.assert_allclose(g - feq, (1 - 1 / tau) * (f - feq), atol=1e-16)
    if tau == 1.0:
        np.testing.assert_allclose(g, feq, atol=1e-16)


def test_streaming_equals_periodic_roll(orc):
    # Pull streaming on a fully periodic lattice is a cyclic shift of each population
    # by its lattice vector: np.roll is an independent implementation of that shift.
    nx, ny, nz = 5, 4, 3
    wl = inp.make_workload("p", nx, ny, nz, 1.0, [None] * 6)
    lat = orc.Lattice.from_workload(wl)
    f = inp.noise(1, (19, nz, ny, nx))
    out = orc.stream(lat, f)
    c, _, _ = orc.lattice()
    for k in range(19):
        ref = np.roll(f[k], shift=(c[k, 2], c[k, 1], c[k, 0]), axis=(0, 1, 2))
        np.testing.assert_array_equal(out[k], ref)


def test_streaming_marks_unknown_sources(orc):
    nx, ny, nz = 5, 4, 6
    wl = inp.make_workload("w", nx, ny, nz, 1.0, [None, None, inp.ZERO, inp.ZERO, inp.ZERO, inp.ZERO])
    lat = orc.Lattice.from_workload(wl)
    f = inp.noise(2, (19, nz, ny, nx))
    out = orc.stream(lat, f)
    c, _, _ = orc.lattice()
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for k in range(19):
        sy, sz = y - c[k, 1], z - c[k, 2]
        outside = (sy < 0) | (sy >= ny) | (sz < 0) | (sz >= nz)
        assert np.isnan(out[k][outside]).all()
        assert not np.isnan(out[k][~outside]).any()
        ref = np.roll(f[k], shift=(c[k, 2], c[k, 1], c[k, 0]), axis=(0, 1, 2))
        np.testing.assert_array_equal(out[k][~outside], ref[~outside])
