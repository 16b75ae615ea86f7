"""GPU parity of solid nodes (mid-grid bounce-back) with the FP64 oracle."""
import numpy as np
import pytest

import lbm_inputs as inp
from lbm_testlib import decode, encode, noisy_state, run_pair, velocity_error

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 5e-3}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def obstacle_duct():
    wl = inp.duct(24, 12, 10, 0.8, 0.05, 30.0)
    r = inp.uniform(91, 5, np.arange(wl.cells)).reshape(wl.nz, wl.ny, wl.nx)
    solid = (r < 0.1).astype(np.uint8)
    solid[:, :, [0, -1]] = 0    # keep the inlet and outlet planes fluid
    wl.solid = solid
    return wl


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("name", ["tilted", "obstacles"])
def test_solid_nodes_match_oracle(name, prec):
    wl = inp.tilted_channel(steps=0) if name == "tilted" else obstacle_duct()
    f0 = noisy_state((19, wl.nz, wl.ny, wl.nx), 70, amp=0.01, u=(0.002, 0.0, 0.004))
    got, ref = run_pair(wl, prec, f0, 30, form=1)
    fluid = wl.solid == 0
    assert velocity_error(wl, got, ref) <= TOL[prec]
    if prec == "f64":
        assert np.abs(got - ref)[:, fluid].max() / np.abs(ref).max() <= 1e-12
    # solid nodes are carried unchanged, bit for bit
    start = decode(encode(f0, prec), prec)
    np.testing.assert_array_equal(got[:, ~fluid], start[:, ~fluid])


def test_solid_nodes_need_the_ab_scheme():
    import paper_0811_4593_gb300 as lbm
    wl = inp.tilted_channel(steps=0)
    with lbm.Lattice(wl.nx, wl.ny, wl.nz, wl.tau, [None] * 4 + wl.utabs[4:], "f32", scheme="aa") as lat:
        with pytest.raises(lbm.LBMError):
            lat.set_solid(wl.solid)
