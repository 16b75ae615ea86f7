"""lbm_reduce_state_static: the state reduction for callers that cannot allocate.

Some users of the library cannot call cudaMalloc at the point where they need a
residual: their device memory is owned by another pool, or they must not trigger the
device-wide synchronisation an allocation or free can cause, or allocation is forbidden
in that code path. lbm_reduce_state_static serves them from a static scratch array
inside the library; every other buffer is theirs.

The test drives it through the C ABI on buffers the test owns and checks it against
lbm_residual (the context-based entry point that computes the same reduction) on two
calls in a row, the second after the state has moved on, so that the velocity snapshot
the first call wrote is what the second one compares against.
"""
import ctypes as C
import math

import pytest

import lbm_inputs as inp
from lbm_testlib import encode, noisy_state

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


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_static_reduction_matches_context_reduction(lbm, prec):
    import torch
    wl = inp.duct(37, 19, 23, 0.8, 0.05, 30.0)  # 16,169 nodes: 64 blocks, ragged tail
    nx, ny, nz = wl.dims
    storage = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16}[prec]
    compute = torch.float64 if prec == "f64" else torch.float32
    pops = torch.empty((19, nz, ny, nx), dtype=storage, device="cuda")
    snap = torch.zeros((3, nz, ny, nx), dtype=compute, device="cuda")
    sums = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    fn = lbm.lib().lbm_reduce_state_static
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(encode(noisy_state((19, nz, ny, nx), 41, u=(0.02, 0.01, 0.0)), prec))
        for call in range(2):
            r_ref, m_ref = lat.residual()
            lat.get_populations(out=pops)
            torch.cuda.synchronize()
            st = fn(C.c_void_p(pops.data_ptr()), nx, ny, nz, PREC_CODE[prec], wl.rho0,
                    C.c_void_p(snap.data_ptr()), C.c_void_p(sums.data_ptr()),
                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert st == 0, lbm.lib().lbm_last_error(None)
            torch.cuda.synchronize()
            s = sums.cpu().numpy()
            r = math.sqrt(s[1]) / math.sqrt(s[2])
            assert s[3] == 0.0
            assert abs(s[0] - m_ref) <= REL_TOL[prec] * abs(m_ref), (call, s[0], m_ref)
            assert abs(r - r_ref) <= REL_TOL[prec] * abs(r_ref), (call, r, r_ref)
            if call == 0:
                assert abs(r - 1.0) < 1e-12  # the first snapshot is zero
            lat.step(5)


def test_static_reduction_rejects_lattices_beyond_its_scratch(lbm):
    import torch
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    st = lbm.lib().lbm_reduce_state_static(p, 257, 256, 256, 1, 1.0, p, p, None)
    assert st == -1
    msg = lbm.lib().lbm_last_error(None).decode()
    assert "16777216" in msg
