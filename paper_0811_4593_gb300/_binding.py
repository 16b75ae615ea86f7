"""ctypes binding to ``liblbm.so`` (C ABI in include/lbm.h).

Argument marshalling only: every step of the solver runs in the CUDA library. PyTorch
provides device memory (the library's allocator hook is pointed at PyTorch's caching
allocator) and streams. There is no CPU fallback: if the library is missing or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the library (the index-checking debug build)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_DIVERGED, LBM_ERR_STATE = 0, -1, -2, -3, -4, -5
PRECISIONS = {"f64": 0, "f32": 1, "f16": 2}
SCHEMES = {"ab": 0, "aa": 1}
STORAGE_DTYPE = {"f64": np.float64, "f32": np.float32, "f16": np.float16}
LBM_HOST, LBM_DEVICE = 0, 1
FACE_PERIODIC, FACE_VELOCITY, FACE_PRESSURE = 0, 1, 2

# Every function the header declares, with its C signature.
EXPORTS = {
    "lbm_set_allocator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_int, C.c_double,
                             C.POINTER(C.c_void_p)]),
    "lbm_create_scheme": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_int, C.c_double,
                                    C.c_int, C.POINTER(C.c_void_p)]),
    "lbm_destroy": (C.c_int, [C.c_void_p]),
    "lbm_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_step_residual": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_residual": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_macros": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_set_populations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "lbm_get_populations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "lbm_sync": (C.c_int, [C.c_void_p]),
    "lbm_set_solid": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_set_geometry": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_set_body_force": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "lbm_check_guards": (C.c_int, [C.c_void_p]),
    "lbm_rule_unknowns": (C.c_int, [C.c_int, C.POINTER(C.c_uint32)]),
    "lbm_debug_bounds_errors": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_uint64)]),
    "lbm_fp64_fma_rate": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_debug_drop_staged_copies": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_info": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_batch_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "lbm_batch_destroy": (C.c_int, [C.c_void_p]),
    "lbm_batch_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_batch_attach": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "lbm_batch_detach": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_batch_step": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "lbm_batch_results": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_batch_info": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_reduce_state_static": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
}


class FaceSpec(C.Structure):
    _fields_ = [("kind", C.c_int), ("u", C.c_double * 3), ("u_table", C.POINTER(C.c_double)),
                ("rho", C.c_double), ("rho_table", C.POINTER(C.c_double))]


class Pressure:
    """A pressure face: prescribed density (scalar or (n2, n1) table) and tangential
    velocity (3-vector or (n2, n1, 3) table; its normal component is ignored)."""

    def __init__(self, rho, u=(0.0, 0.0, 0.0)):
        self.rho = rho
        self.u = u


class Info(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("precision", C.c_int),
                ("steps", C.c_int64), ("kernel_launches", C.c_int64), ("bytes_per_update", C.c_int64),
                ("device_bytes", C.c_int64), ("scheme", C.c_int)]


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lbm status {status}: {message}")
        self.status = status


class LBMDiverged(LBMError):
    def __init__(self, status, message, residual=float("nan"), mass=float("nan")):
        super().__init__(status, message)
        self.residual = residual
        self.mass = mass


_lib = None
_lock = threading.Lock()
_hooks = None


def library_path() -> str:
    return LIB_PATH


def debug_bounds_errors():
    """(enabled, count): whether the loaded library is the index-checking debug build,
    and the out-of-range indices its sweeps met since the last call."""
    en, n = C.c_int(), C.c_uint64()
    check(lib().lbm_debug_bounds_errors(C.byref(en), C.byref(n)))
    return bool(en.value), int(n.value)


def fp64_fma_rate(iters: int = 20000):
    """(thread-level FP64 FMAs per second, milliseconds of the timed launch) of the
    current device, from lbm_fp64_fma_rate."""
    r, ms = C.c_double(), C.c_double()
    check(lib().lbm_fp64_fma_rate(int(iters), C.byref(r), C.byref(ms)))
    return r.value, ms.value


def lib():
    """Load liblbm.so, raising if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built: run `python -m paper_0811_4593_gb300.build` "
                                   f"(needs nvcc)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in EXPORTS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error(ctx=None) -> str:
    msg = lib().lbm_last_error(ctx)
    return msg.decode() if msg else ""


def check(status: int, ctx=None):
    if status != LBM_OK:
        raise LBMError(status, last_error(ctx))


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _hooks
    import torch
    if _hooks is not None:
        return
    ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
    FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

    def _alloc(nbytes, _user):
        try:
            dev = torch.cuda.current_device()
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch.cuda.current_stream(dev)))
        except Exception:  # noqa: BLE001 - an allocation failure is reported to C as NULL
            return None

    def _free(ptr, _user):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC(_alloc), FREE(_free)
    check(lib().lbm_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None))
    _hooks = (a, f)


def use_default_allocator():
    global _hooks
    check(lib().lbm_set_allocator(None, None, None))
    _hooks = None


def _face_specs(nx, ny, nz, faces):
    """faces[i]: None (periodic), a velocity 3-vector or (n2, n1, 3) table, or a
    Pressure."""
    specs = (FaceSpec * 6)()
    keep = []
    dims = (nx, ny, nz)
    for i, fu in enumerate(faces):
        if fu is None:
            specs[i].kind = FACE_PERIODIC
            continue
        a = i // 2
        t1, t2 = [b for b in range(3) if b != a]
        shape2 = (dims[t2], dims[t1])
        if isinstance(fu, Pressure):
            specs[i].kind = FACE_PRESSURE
            rho = np.asarray(fu.rho, np.float64)
            if rho.shape == ():
                specs[i].rho = float(rho)
            else:
                if rho.shape != shape2:
                    raise ValueError(f"face {i}: density table shape {rho.shape}, expected {shape2}")
                rho = np.ascontiguousarray(rho)
                keep.append(rho)
                specs[i].rho_table = rho.ctypes.data_as(C.POINTER(C.c_double))
            fu = fu.u
        else:
            specs[i].kind = FACE_VELOCITY
        arr = np.asarray(fu, np.float64)
        if arr.shape == (3,):
            for j in range(3):
                specs[i].u[j] = float(arr[j])
        else:
            if arr.shape != shape2 + (3,):
                raise ValueError(f"face {i}: table shape {arr.shape}, expected {shape2 + (3,)}")
            arr = np.ascontiguousarray(arr)
            keep.append(arr)
            specs[i].u_table = arr.ctypes.data_as(C.POINTER(C.c_double))
    return specs, keep


class Lattice:
    """One D3Q19 lattice resident on the current CUDA device.

    ``faces`` lists the six faces (x=0, x=nx-1, y=0, y=ny-1, z=0, z=nz-1); each is None
    (periodic), a velocity 3-vector, a table of prescribed velocities (n2, n1, 3), or a
    Pressure (prescribed density and tangential velocity).
    ``precision`` is "f64" (f stored as double), "f32" or "f16" (f - w rho0 stored as
    float or binary16). ``scheme`` is "ab" (two arrays) or "aa" (one array, steps in
    pairs).
    """

    def __init__(self, nx, ny, nz, tau, faces, precision="f32", rho0=1.0, stream=None,
                 torch_allocator=True, scheme="ab"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the lattice runs only on the GPU")
        if torch_allocator:
            use_torch_allocator()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.tau, self.rho0 = float(tau), float(rho0)
        self.precision = precision
        self.scheme = scheme
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        specs, keep = _face_specs(self.nx, self.ny, self.nz, faces)
        out = C.c_void_p()
        st = lib().lbm_create_scheme(self.nx, self.ny, self.nz, self.tau, C.cast(specs, C.c_void_p),
                                     PRECISIONS[precision], self.rho0, SCHEMES[scheme], C.byref(out))
        del keep
        check(st)
        self._ctx = out
        check(lib().lbm_set_stream(self._ctx, C.c_void_p(self.stream.cuda_stream)), self._ctx)

    def set_solid(self, solid):
        """Mark solid nodes (uint8 (nz, ny, nx), nonzero = solid): mid-grid bounce-back
        walls; A/B scheme only."""
        m = np.ascontiguousarray(solid, np.uint8)
        if m.shape != (self.nz, self.ny, self.nx):
            raise ValueError(f"solid mask shape {m.shape} != {(self.nz, self.ny, self.nx)}")
        check(lib().lbm_set_solid(self.ctx, C.c_void_p(m.ctypes.data)), self.ctx)

    def set_geometry(self, solid=None, code=None):
        """General geometry: solid nodes (uint8, nonzero = solid) and on-site rule codes
        (int8, the normal as a lattice-vector index; see lbm_set_geometry), both
        (nz, ny, nx) or None; A/B scheme only."""
        shape = (self.nz, self.ny, self.nx)
        m = None if solid is None else np.ascontiguousarray(solid, np.uint8)
        c = None if code is None else np.ascontiguousarray(code, np.int8)
        for name, a in (("solid", m), ("code", c)):
            if a is not None and a.shape != shape:
                raise ValueError(f"{name} shape {a.shape} != {shape}")
        check(lib().lbm_set_geometry(self.ctx, None if m is None else C.c_void_p(m.ctypes.data),
                                     None if c is None else C.c_void_p(c.ctypes.data)), self.ctx)

    def set_body_force(self, force):
        """Uniform body force F (eq. gravity); A/B scheme only."""
        f = (C.c_double * 3)(*[float(v) for v in force])
        check(lib().lbm_set_body_force(self.ctx, f), self.ctx)

    @classmethod
    def from_workload(cls, wl, precision="f32", **kw):
        """A lattice for any object with nx, ny, nz, tau, rho0, kinds, utabs (and ptabs
        for pressure faces, solid / code for a geometry, force for a body force)."""
        ptabs = getattr(wl, "ptabs", None) or [None] * 6
        faces = []
        for k, t, p in zip(wl.kinds, wl.utabs, ptabs):
            if k == FACE_PERIODIC:
                faces.append(None)
            elif k == FACE_PRESSURE:
                faces.append(Pressure(p, t))
            else:
                faces.append(t)
        lat = cls(wl.nx, wl.ny, wl.nz, wl.tau, faces, precision, wl.rho0, **kw)
        solid, code = getattr(wl, "solid", None), getattr(wl, "code", None)
        if code is not None:
            lat.set_geometry(solid, code)
        elif solid is not None:
            lat.set_solid(solid)
        if getattr(wl, "force", None) is not None:
            lat.set_body_force(wl.force)
        return lat

    def check_guards(self):
        """Raise LBMError if a write landed just outside one of the lattice's buffers."""
        check(lib().lbm_check_guards(self.ctx), self.ctx)

    # -- lifetime -------------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            ctx, self._ctx = self._ctx, None
            try:
                if os.environ.get("LBM_CHECK_GUARDS") == "1":
                    check(lib().lbm_check_guards(ctx), ctx)
            finally:
                lib().lbm_destroy(ctx)

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def ctx(self):
        if not self._ctx:
            raise RuntimeError("lattice is closed")
        return self._ctx

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (19, self.nz, self.ny, self.nx)

    # -- time stepping --------------------------------------------------------------
    def step(self, n: int = 1):
        check(lib().lbm_step(self.ctx, int(n)), self.ctx)

    def _reduced(self, st, r, m):
        if st == LBM_ERR_DIVERGED:
            raise LBMDiverged(st, last_error(self.ctx), r.value, m.value)
        check(st, self.ctx)
        return r.value, m.value

    def step_residual(self, n: int):
        r, m = C.c_double(), C.c_double()
        st = lib().lbm_step_residual(self.ctx, int(n), C.byref(r), C.byref(m))
        return self._reduced(st, r, m)

    def residual(self):
        r, m = C.c_double(), C.c_double()
        st = lib().lbm_residual(self.ctx, C.byref(r), C.byref(m))
        return self._reduced(st, r, m)

    def sync(self):
        check(lib().lbm_sync(self.ctx), self.ctx)

    # -- data -----------------------------------------------------------------------
    def macros(self, rho=None, u=None):
        """(rho[nz,ny,nx], u[3,nz,ny,nx]) as torch tensors on the lattice's device."""
        import torch
        dt = torch.float64 if self.precision == "f64" else torch.float32
        if rho is None:
            rho = torch.empty((self.nz, self.ny, self.nx), dtype=dt, device=self.device)
        if u is None:
            u = torch.empty((3, self.nz, self.ny, self.nx), dtype=dt, device=self.device)
        for t in (rho, u):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"macros buffers must be contiguous {dt} CUDA tensors")
        check(lib().lbm_macros(self.ctx, C.c_void_p(rho.data_ptr()), C.c_void_p(u.data_ptr())), self.ctx)
        return rho, u

    def set_populations(self, f, z0: int = 0):
        """Load planes z0.. of the state from an array [19][nzs][ny][nx] in the storage
        dtype (float64 holds f; float32 and float16 hold f - w rho0); a numpy array is
        read from host memory, a CUDA tensor from device memory."""
        nzs = int(f.shape[1])
        self._check_pop_shape(f, nzs)
        if isinstance(f, np.ndarray):
            a = np.ascontiguousarray(f, STORAGE_DTYPE[self.precision])
            check(lib().lbm_set_populations(self.ctx, C.c_void_p(a.ctypes.data), int(z0), nzs, LBM_HOST),
                  self.ctx)
        else:
            t = f.contiguous()
            check(lib().lbm_set_populations(self.ctx, C.c_void_p(t.data_ptr()), int(z0), nzs,
                                            LBM_HOST if not t.is_cuda else LBM_DEVICE), self.ctx)

    def get_populations(self, z0: int = 0, nzs: int | None = None, out=None):
        """Planes z0..z0+nzs-1 of the state as a host numpy array (or into ``out``)."""
        nzs = self.nz - z0 if nzs is None else int(nzs)
        if out is None:
            out = np.empty((19, nzs, self.ny, self.nx), STORAGE_DTYPE[self.precision])
        self._check_pop_shape(out, nzs)
        if isinstance(out, np.ndarray):
            check(lib().lbm_get_populations(self.ctx, C.c_void_p(out.ctypes.data), int(z0), nzs, LBM_HOST),
                  self.ctx)
        else:
            check(lib().lbm_get_populations(self.ctx, C.c_void_p(out.data_ptr()), int(z0), nzs,
                                            LBM_HOST if not out.is_cuda else LBM_DEVICE), self.ctx)
        return out

    def _check_pop_shape(self, a, nzs):
        if tuple(a.shape) != (19, nzs, self.ny, self.nx):
            raise ValueError(f"population array shape {tuple(a.shape)} != {(19, nzs, self.ny, self.nx)}")

    def info(self) -> dict:
        i = Info()
        check(lib().lbm_info(self.ctx, C.byref(i)), self.ctx)
        return {f: getattr(i, f) for f, _ in Info._fields_}


class BatchInfo(C.Structure):
    _fields_ = [("capacity", C.c_int), ("attached", C.c_int), ("grid", C.c_int), ("nodes", C.c_int64),
                ("steps", C.c_int64), ("kernel_launches", C.c_int64), ("device_bytes", C.c_int64)]


class Batch:
    """Slots of resident lattices advanced together by one persistent launch per step
    (CUDA-graph replays of the n-step loop). Attach Lattice objects of the batch's
    precision; results of residual steps come back per slot."""

    NO_RESULT = 1

    def __init__(self, capacity: int, precision: str = "f32", stream=None, torch_allocator=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: batches run only on the GPU")
        if torch_allocator:
            use_torch_allocator()
        self.capacity = int(capacity)
        self.precision = precision
        out = C.c_void_p()
        st = lib().lbm_batch_create(self.capacity, PRECISIONS[precision], C.byref(out))
        if st != LBM_OK:
            raise LBMError(st, lib().lbm_batch_last_error(None).decode())
        self._b = out
        self.lattices = [None] * self.capacity
        if stream is not None:
            self._check(lib().lbm_batch_set_stream(self._b, C.c_void_p(stream.cuda_stream)))
        self._r = (C.c_double * self.capacity)()
        self._m = (C.c_double * self.capacity)()
        self._s = (C.c_int * self.capacity)()

    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, lib().lbm_batch_last_error(self._b).decode())

    def close(self):
        if getattr(self, "_b", None):
            lib().lbm_batch_destroy(self._b)
            self._b = None
            self.lattices = [None] * self.capacity

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def attach(self, slot: int, lattice: "Lattice"):
        self._check(lib().lbm_batch_attach(self._b, int(slot), lattice.ctx))
        self.lattices[slot] = lattice

    def detach(self, slot: int):
        self._check(lib().lbm_batch_detach(self._b, int(slot)))
        self.lattices[slot] = None

    def free_slots(self):
        return [i for i, l in enumerate(self.lattices) if l is None]

    def step(self, n: int, residual: bool = False):
        self._check(lib().lbm_batch_step(self._b, int(n), 1 if residual else 0))

    def results(self):
        """[(residual, mass, status)] per slot; status 0 ok, -4 diverged, 1 no result."""
        self._check(lib().lbm_batch_results(self._b, self._r, self._m, self._s))
        return [(self._r[i], self._m[i], self._s[i]) for i in range(self.capacity)]

    def info(self) -> dict:
        i = BatchInfo()
        self._check(lib().lbm_batch_info(self._b, C.byref(i)))
        return {f: getattr(i, f) for f, _ in BatchInfo._fields_}
