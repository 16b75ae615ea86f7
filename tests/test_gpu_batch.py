"""GPU tests of the multi-lattice batch (persistent launch + CUDA-graph replay).

A lattice advanced inside a batch must evolve to exactly the bits it reaches when
stepped alone (same per-node code, same grouping of the residual sums), whatever the
other lattices are and however the membership changes between replays; and a mixed
batch must match the FP64 oracle lattice by lattice.
"""
import numpy as np
import pytest

import lbm_inputs as inp
from lbm_testlib import decode, encode, noisy_state, velocity_error

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def mix():
    """Lattices of different sizes, boundary types and relaxation times (ragged node
    counts, so block boundaries fall inside rows)."""
    return [
        inp.duct(37, 19, 23, 0.8, 0.05, 30.0),
        inp.channel(33, 20, 21, 0.7, (0.04, 0.01, 0.0)),
        inp.random_face_workload(5, 11, 9, 7, 1.2, (False, True, False)),
        inp.couette(),
        inp.duct(64, 16, 16, 0.6, 0.03, 15.0),
    ]


def start(wl, prec, seed):
    import paper_0811_4593_gb300 as lbm
    lat = lbm.Lattice.from_workload(wl, prec)
    lat.set_populations(encode(noisy_state((19, wl.nz, wl.ny, wl.nx), seed, u=(0.01, 0.005, -0.004)), prec))
    return lat


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_batched_lattices_match_solo_runs_bitwise(prec):
    import paper_0811_4593_gb300 as lbm
    wls = mix()
    solo = []
    for i, wl in enumerate(wls):
        with start(wl, prec, 10 + i) as lat:
            lat.step(9)
            r, m = lat.step_residual(1)
            lat.step(4)
            r2, m2 = lat.step_residual(6)
            solo.append((lat.get_populations(), (r, m), (r2, m2)))
    with lbm.Batch(8, prec) as b:
        lats = [start(wl, prec, 10 + i) for i, wl in enumerate(wls)]
        slots = [0, 2, 4, 6, 7]
        for lat, slot in zip(lats, slots):
            b.attach(slot, lat)
        b.step(10, residual=True)
        res1 = b.results()
        b.step(10, residual=True)
        res2 = b.results()
        for i, lat in enumerate(lats):
            np.testing.assert_array_equal(lat.get_populations(), solo[i][0])
            assert res1[slots[i]][:2] == solo[i][1]
            assert res2[slots[i]][:2] == solo[i][2]
            assert res1[slots[i]][2] == 0
        info = b.info()
        assert info["attached"] == len(lats)
        assert info["steps"] == 20
        for lat in lats:
            lat.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_mixed_batch_matches_oracle(prec):
    import oracle
    import paper_0811_4593_gb300 as lbm
    wls = mix()[:4]
    steps = 24
    with lbm.Batch(4, prec) as b:
        lats = []
        for i, wl in enumerate(wls):
            lat = start(wl, prec, 30 + i)
            lats.append(lat)
            b.attach(i, lat)
        b.step(steps)
        for i, wl in enumerate(wls):
            got = decode(lats[i].get_populations(), prec)
            s0 = encode(noisy_state((19, wl.nz, wl.ny, wl.nx), 30 + i, u=(0.01, 0.005, -0.004)), prec)
            ref = oracle.run(oracle.Lattice.from_workload(wl), decode(s0, prec), steps)
            assert velocity_error(wl, got, ref) <= TOL[prec]
        for lat in lats:
            lat.close()


def test_membership_changes_between_graph_replays():
    import paper_0811_4593_gb300 as lbm
    prec = "f32"
    wls = mix()
    # A stays for 10 + 10 + 10 + 7 steps, B leaves after 20, C joins B's slot for 17
    ref = {}
    for name, i, n in (("A", 0, 37), ("B", 1, 20), ("C", 2, 17)):
        with start(wls[i], prec, 50 + i) as lat:
            lat.step(n)
            ref[name] = lat.get_populations()
    with lbm.Batch(3, prec) as b:
        A, B = start(wls[0], prec, 50), start(wls[1], prec, 51)
        b.attach(0, A)
        b.attach(1, B)
        b.step(10)
        b.step(10)           # graph replay with the same membership
        b.detach(1)
        np.testing.assert_array_equal(B.get_populations(), ref["B"])
        C = start(wls[2], prec, 52)
        b.attach(1, C)       # same slot, another lattice
        b.step(10)           # replay with a rewritten table
        b.step(7)            # odd count: another graph, parity bookkeeping
        np.testing.assert_array_equal(C.get_populations(), ref["C"])
        np.testing.assert_array_equal(A.get_populations(), ref["A"])
        b.detach(0)
        A.step(3)            # a detached lattice steps alone again
        with start(wls[0], prec, 50) as lat:
            lat.step(40)
            np.testing.assert_array_equal(A.get_populations(), lat.get_populations())
        for lat in (A, B, C):
            lat.close()


def test_results_status_per_slot():
    import paper_0811_4593_gb300 as lbm
    prec = "f32"
    slab = inp.make_workload("slab", 8, 10, 10, 0.55, [None, None, None, None, inp.ZERO, inp.ZERO])
    with lbm.Batch(4, prec) as b:
        good = start(inp.duct(20, 9, 9, 0.9, 0.05, 30.0), prec, 61)
        bad = lbm.Lattice.from_workload(slab, prec)
        bad.set_populations(encode(noisy_state((19, 10, 10, 8), 3, amp=1e-3), prec))
        b.attach(0, good)
        b.attach(3, bad)
        status = None
        for _ in range(40):
            b.step(250, residual=True)
            res = b.results()
            status = [s for _, _, s in res]
            if status[3] == -4:
                break
        assert status[3] == -4
        assert status[0] == 0
        assert status[1] == 1 and status[2] == 1
        good.close()
        bad.close()


def test_attach_rules():
    import paper_0811_4593_gb300 as lbm
    with lbm.Batch(2, "f32") as b, lbm.Batch(2, "f32") as b2:
        a = start(inp.couette(), "f32", 1)
        c = start(inp.couette(), "f64", 1)
        b.attach(0, a)
        with pytest.raises(lbm.LBMError):
            b.attach(0, start(inp.couette(), "f32", 2))   # occupied
        with pytest.raises(lbm.LBMError):
            b2.attach(0, a)                              # already attached
        with pytest.raises(lbm.LBMError):
            b.attach(1, c)                               # precision differs
        with pytest.raises(lbm.LBMError):
            b.attach(5, c)                               # slot out of range
        a.step(3)                                        # own calls wait for the batch
        b.step(2)
        a.close()                                        # destroy detaches
        assert b.info()["attached"] == 0
        b.step(2)                                        # empty batch: no-op
        c.close()


def test_injected_nan_is_reported_per_lattice():
    # a host-built state with one non-finite population: the next residual step reports
    # the lattice as diverged, alone and in a batch, without touching its neighbours
    import paper_0811_4593_gb300 as lbm
    wl = inp.duct(20, 9, 9, 0.9, 0.05, 30.0)
    bad_state = encode(noisy_state((19, wl.nz, wl.ny, wl.nx), 5), "f32")
    bad_state[3, 4, 4, 10] = np.nan
    with start(wl, "f32", 5) as lat:
        lat.set_populations(bad_state)
        with pytest.raises(lbm.LBMDiverged):
            lat.step_residual(1)
    with lbm.Batch(3, "f32") as b:
        good = start(wl, "f32", 6)
        bad = start(wl, "f32", 7)
        bad.set_populations(bad_state)
        b.attach(0, good)
        b.attach(2, bad)
        b.step(1, residual=True)
        status = [s for _, _, s in b.results()]
        assert status == [0, 1, -4]
        good.close()
        bad.close()
