"""GPU parity on the benchmark configurations at their stated sizes: the 256 x 64 x 64
square duct (tilted parabolic inlet and outlet, resting walls, tau 0.6 and 1.0; at tau
0.6 also in one array with AA streaming) and the plane Poiseuille sweep (4 x 4 x Lz,
parabolic inlet and outlet of peak 0.02), each run from rest for a few hundred to a few
thousand steps on the GPU and in the FP64 oracle, compared node by node (velocity error
in units of the largest velocity).

Bars: FP64 1e-12, FP32 1e-5; binary16 storage at about twice the error measured for
each case on a GB300 (duct 5.2e-4 / 4.4e-4 at tau 0.6 / 1.0; Poiseuille 4.2e-4, 2.9e-4,
1.3e-3 at Lz 16, 64, 256 and 2.8e-4 at Lz 64, tau 1.5).
"""
import numpy as np
import pytest

import lbm_inputs as inp

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
# binary16: the duct after 300 steps, Poiseuille after 3000
F16_TOL = {("duct", 0.6): 1.1e-3, ("duct", 1.0): 9e-4,
           ("poiseuille", 16, 1.0): 9e-4, ("poiseuille", 64, 1.0): 6e-4, ("poiseuille", 256, 1.0): 2.6e-3,
           ("poiseuille", 64, 1.5): 6e-4}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def gpu_and_oracle(wl, prec, steps, scheme="ab"):
    import oracle
    import paper_0811_4593_gb300 as lbm
    olat = oracle.Lattice.from_workload(wl)
    ref = oracle.run(olat, oracle.init_equilibrium(olat), steps)
    _, uo = oracle.macros(olat, ref)
    with lbm.Lattice.from_workload(wl, prec, scheme=scheme) as lat:
        lat.step(steps)
        _, u = lat.macros()
        u = u.double().cpu().numpy()
    return float(np.abs(u - uo).max() / np.abs(uo).max())


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("tau", [0.6, 1.0])
def test_duct_256x64x64_against_oracle(prec, tau):
    err = gpu_and_oracle(inp.duct(256, 64, 64, tau, 0.05, 30.0), prec, 300)
    print(f"duct tau {tau} {prec}: {err:.3e}")
    assert err <= (F16_TOL[("duct", tau)] if prec == "f16" else TOL[prec]), err


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_duct_256x64x64_aa_against_oracle(prec):
    """The same duct in one array (AA streaming): the binary16 lattice runs the row-staged
    AA steps (256-node rows), whose pushes test each population for a target beyond the
    walled y and z faces on the wall rows."""
    err = gpu_and_oracle(inp.duct(256, 64, 64, 0.6, 0.05, 30.0), prec, 300, scheme="aa")
    print(f"duct AA tau 0.6 {prec}: {err:.3e}")
    assert err <= (F16_TOL[("duct", 0.6)] if prec == "f16" else TOL[prec]), err


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("lz,tau", [(16, 1.0), (64, 1.0), (256, 1.0), (64, 1.5)])
def test_plane_poiseuille_against_oracle(prec, lz, tau):
    err = gpu_and_oracle(inp.poiseuille(lz, tau, 0.02), prec, 3000)
    print(f"poiseuille Lz {lz} tau {tau} {prec}: {err:.3e}")
    assert err <= (F16_TOL[("poiseuille", lz, tau)] if prec == "f16" else TOL[prec]), err
