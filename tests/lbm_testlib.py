"""Helpers shared by the GPU parity tests: storage encoding of test states, paired
GPU / oracle runs, error measures. Test infrastructure only."""
from __future__ import annotations

import numpy as np

import lbm_inputs as inp


def weights():
    import oracle
    return oracle.lattice()[1]


def noisy_state(shape, seed, amp=0.02, rho0=1.0, u=(0.0, 0.0, 0.0)):
    """f = f_eq(rho0, u) * (1 + amp * noise), the noise from the shared generator."""
    import oracle
    base = oracle.feq(rho0, u)
    return base[:, None, None, None] * (1.0 + amp * inp.noise(seed, shape))


def encode(f, prec, rho0=1.0):
    """FP64 populations -> the storage array of a precision."""
    if prec == "f64":
        return np.ascontiguousarray(f, np.float64)
    w = weights()
    h = f - (w * rho0)[:, None, None, None]
    return np.ascontiguousarray(h, np.float32 if prec == "f32" else np.float16)


def decode(s, prec, rho0=1.0):
    """Storage array -> FP64 populations."""
    if prec == "f64":
        return s.astype(np.float64)
    w = weights()
    return s.astype(np.float64) + (w * rho0)[:, None, None, None]


def run_pair(wl, prec, f0, steps, form=0):
    """Run `steps` on the GPU and in the oracle from the same stored initial state.
    Returns (gpu populations, oracle populations) as FP64 arrays."""
    import oracle
    import paper_0811_4593_gb300 as lbm
    s0 = encode(f0, prec, wl.rho0)
    with lbm.Lattice.from_workload(wl, prec) as lat:
        lat.set_populations(s0)
        lat.step(steps)
        got = decode(lat.get_populations(), prec, wl.rho0)
    olat = oracle.Lattice.from_workload(wl)
    ref = oracle.run(olat, decode(s0, prec, wl.rho0), steps, form)
    return got, ref


def velocity_error(wl, got, ref):
    """max |u_gpu - u_ref| / max |u_ref| over all nodes (velocities from the oracle's
    moment routine applied to both states)."""
    import oracle
    olat = oracle.Lattice.from_workload(wl)
    _, ug = oracle.macros(olat, got)
    _, ur = oracle.macros(olat, ref)
    scale = max(np.abs(ur).max(), 1e-300)
    return float(np.abs(ug - ur).max() / scale)


def population_error(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def separable_state_slab(tables, nx, ny, z0, z1, amp, prec, rho0=1.0):
    """Storage array of planes z0..z1-1 of the large-lattice test state
    f = w rho0 (1 + amp * eps) with eps from lbm_inputs.separable_noise_slab."""
    w = weights()
    eps = inp.separable_noise_slab(tables, nx, ny, z0, z1)
    f = (w * rho0)[:, None, None, None] * (1.0 + amp * eps)
    return encode(f, prec, rho0)


def separable_value_at(tables, nx, ny, nz, idx, amp, prec, rho0=1.0):
    """The same state, as stored and decoded to FP64, at flat indices k*N + node."""
    w = weights()
    idx = np.asarray(idx, np.int64)
    k = idx // (nx * ny * nz)
    eps = inp.separable_noise_at(tables, nx, ny, nz, idx)
    wr = w[k] * rho0
    f = wr * (1.0 + amp * eps)
    if prec == "f64":
        return f
    return (f - wr).astype(np.float32 if prec == "f32" else np.float16).astype(np.float64) + wr
