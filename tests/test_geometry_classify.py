"""Host-side checks of the geometry classifier (no GPU): the library's rule sets agree
with the oracle's independent ones, the classifier reproduces the codes the workload
generators build analytically, and the codes it gives a voxel sphere pass the oracle's
geometry check (nodes no rule covers fall back to mid-grid bounce-back)."""
import numpy as np
import pytest

import lbm_inputs as inp


@pytest.fixture(scope="module")
def geo():
    from paper_0811_4593_gb300 import build
    build.build()
    from paper_0811_4593_gb300 import geometry
    return geometry


def test_library_rule_sets_equal_the_oracle_ones(geo, orc):
    for code in geo.CODES:
        mask = geo.rule_unknowns(code)
        lib_set = np.array([(mask >> k) & 1 for k in range(19)], bool)
        np.testing.assert_array_equal(lib_set, orc.rule_unknowns(code), err_msg=str(code))
    import paper_0811_4593_gb300 as lbm
    for bad in (0, 51, -6, 127, -19):
        with pytest.raises(lbm.LBMError):
            geo.rule_unknowns(bad)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_classifier_reproduces_the_pillar_codes(geo, axis):
    flow = [a for a in range(3) if a != axis][0]
    wl = inp.pillar_channel(axis=axis, flow=flow)
    walled = [a == axis for a in range(3)]
    np.testing.assert_array_equal(geo.classify(wl.solid, walled), wl.code)


def test_classifier_reproduces_embedded_walls(geo):
    box = inp.make_workload("box", 9, 7, 6, 0.8, [inp.ZERO] * 6)
    emb = inp.embedded_walls(box)
    np.testing.assert_array_equal(geo.classify(emb.solid, (True, True, True)), emb.code)


def sphere(n=(32, 24, 24), r=5.2):
    z, y, x = np.meshgrid(*[np.arange(k) for k in n[::-1]], indexing="ij")
    c = [(k - 1) / 2.0 for k in n]
    return (((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) < r * r).astype(np.uint8)


def test_sphere_codes_pass_the_oracle_check(geo, orc):
    solid = sphere()
    codes = geo.classify(solid, (False, False, False))
    wl = inp.make_workload("sphere", 32, 24, 24, 0.8, [None] * 6)
    wl.solid, wl.code = solid, codes
    assert orc.check_geometry(orc.Lattice.from_workload(wl)) == -1
    assert (codes != 0).sum() > 400
    import paper_0811_4593_gb300 as lbm
    with pytest.raises(lbm.LBMError, match="fit equally"):
        geo.classify(solid, (False, False, False), on_missing="raise")
