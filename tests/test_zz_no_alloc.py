"""lbm_reduce_state_static: the state reduction for callers that cannot allocate.

Some users of the library cannot call cudaMalloc at the point where they need a
residual: their device memory is owned by another pool, or they must not trigger the
device-wide synchronisation an allocation or free can cause, or allocation is forbidden
in that code path. lbm_reduce_state_static serves them from a static scratch array
inside the library; every other buffer is theirs.

The tests drive it through the C ABI on buffers the test owns, on two calls in a row
(the second after the state has moved on, so that the velocity snapshot the first call
wrote is what the second one compares against), and check each call
  * against the FP64 oracle's reduction of the same stored populations: mass,
    sum |u - u_prev|^2, sum |u|^2 and the bad-node count, with u_prev the oracle's
    velocities of the previous state, and the velocity snapshot the call writes back
    against the oracle's velocities;
  * against lbm_residual, the context-based entry point of the same reduction.
This file is collected last, so that a run stopping at its first failure has already
run every other test.
"""
import ctypes as C
import math

import numpy as np
import pytest

import lbm_inputs as inp
from lbm_testlib import decode, encode, noisy_state

pytestmark = pytest.mark.gpu

PREC_CODE = {"f64": 0, "f32": 1, "f16": 2}
REL_TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 1e-5}


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    from paper_0811_4593_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    import paper_0811_4593_gb300 as lbm
    return lbm


def static_reduce(lbm, pops, dims, prec, rho0, snap, sums):
    import torch
    nx, ny, nz = dims
    st = lbm.lib().lbm_reduce_state_static(C.c_void_p(pops.data_ptr()), nx, ny, nz, PREC_CODE[prec], rho0,
                                           C.c_void_p(snap.data_ptr()), C.c_void_p(sums.data_ptr()),
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lbm.lib().lbm_last_error(None)
    torch.cuda.synchronize()
    return sums.cpu().numpy().copy()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_static_reduction_matches_oracle_and_context_reduction(lbm, prec):
    import torch

    import oracle
    wl = inp.duct(37, 19, 23, 0.8, 0.05, 30.0)  # 16,169 nodes: 64 blocks, ragged tail
    nx, ny, nz = wl.dims
    olat = oracle.Lattice.from_workload(wl)
    storage = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16}[prec]
    compute = torch.float64 if prec == "f64" else torch.float32
    pops = torch.empty((19, nz, ny, nx), dtype=storage, device="cuda")
    snap = torch.zeros((3, nz, ny, nx), dtype=compute, device="cuda")
    sums = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    rtol = REL_TOL[prec]
    u_prev = None
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(encode(noisy_state((19, nz, ny, nx), 41, u=(0.02, 0.01, 0.0)), prec))
        for call in range(2):
            r_ctx, m_ctx = lat.residual()
            lat.get_populations(out=pops)
            torch.cuda.synchronize()
            s = static_reduce(lbm, pops, wl.dims, prec, wl.rho0, snap, sums)
            # the oracle on the decoded stored populations
            f = decode(pops.cpu().numpy(), prec, wl.rho0)
            red = oracle.reduce(olat, f, u_prev)
            assert s[0] == pytest.approx(red[0], rel=rtol), (call, s[0], red[0])
            assert s[2] == pytest.approx(red[2], rel=rtol), (call, s[2], red[2])
            # sum |u - u_prev|^2: the float snapshot carries rounding of order 1e-7 |u|,
            # so its error is bounded in units of sum |u|^2
            assert abs(s[1] - red[1]) <= rtol * red[2], (call, s[1], red[1])
            assert s[3] == red[3] == 0.0
            _, u = oracle.macros(olat, f)
            atol = (1e-12 if prec == "f64" else 1e-6) * np.abs(u).max()
            np.testing.assert_allclose(snap.double().cpu().numpy(), u, rtol=0, atol=atol)
            u_prev = u
            # the context entry point on the same state
            r = math.sqrt(s[1]) / math.sqrt(s[2])
            assert abs(s[0] - m_ctx) <= rtol * abs(m_ctx), (call, s[0], m_ctx)
            assert abs(r - r_ctx) <= rtol * abs(r_ctx), (call, r, r_ctx)
            if call == 0:
                assert abs(r - 1.0) < 1e-12  # the first snapshot is zero
            lat.step(5)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_static_reduction_counts_bad_nodes_like_the_oracle(lbm, prec):
    import torch

    import oracle
    nx, ny, nz = 29, 11, 7          # 2,233 nodes: 9 blocks, ragged tail
    olat = oracle.Lattice(nx, ny, nz, [0] * 6, [None] * 6, 1.0)
    f = noisy_state((19, nz, ny, nx), 43, u=(0.01, 0.0, -0.01))
    stored = encode(f, prec)
    stored[3, 2, 5, 17] = np.nan                    # one non-finite population
    stored[:, 6, 10, 28] = -0.2                     # density 1 - 19 * 0.2 < 0 (shifted)
    if prec == "f64":
        stored[:, 6, 10, 28] = -0.01                # density -0.19
    stored[[0, 7, 12], 0, 0, 0] = np.inf            # several bad populations: one node
    pops = torch.from_numpy(stored).cuda()
    snap = torch.zeros((3, nz, ny, nx), dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")
    sums = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    s = static_reduce(lbm, pops, (nx, ny, nz), prec, 1.0, snap, sums)
    red = oracle.reduce(olat, decode(stored, prec), None)
    assert s[3] == red[3] == 3.0, (s, red)


def test_static_reduction_rejects_lattices_beyond_its_scratch(lbm):
    import torch
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    st = lbm.lib().lbm_reduce_state_static(p, 257, 256, 256, 1, 1.0, p, p, None)
    assert st == -1
    msg = lbm.lib().lbm_last_error(None).decode()
    assert "16777216" in msg
