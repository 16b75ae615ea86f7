"""FP64 CPU oracle for the D3Q19 BGK solver with the on-site velocity boundary
condition of Hecht & Harting (arXiv:0811.4593).

TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline leg
of the benchmark may import this package. It wraps ``liblbm_oracle.so`` (plain C,
``lbm_oracle.c``) with numpy arrays and shares no code with the CUDA library.

Array conventions: populations are ``float64`` arrays of shape ``(19, nz, ny, nx)``;
index ``k`` holds the paper's population ``f_{k+1}``. Faces are numbered
0: x=0, 1: x=nx-1, 2: y=0, 3: y=ny-1, 4: z=0, 5: z=nz-1.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

Q = 19
_LIB = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_feq.argtypes = [C.c_double, _dp, _dp]
        L.orc_moments.argtypes = [_dp, _dp]
        L.orc_collide.argtypes = [_dp, C.c_double]
        L.orc_close_face.argtypes = [C.c_int, C.c_int, _dp, _dp, C.POINTER(C.c_double)]
        L.orc_close_edge.argtypes = [C.c_int, C.c_int, _dp, C.c_double]
        L.orc_close_corner.argtypes = [C.c_int, C.c_int, C.c_int, _dp, C.c_double]
        L.orc_close_face_pressure.argtypes = [C.c_int, C.c_int, _dp, C.c_double, _dp, C.POINTER(C.c_double)]
        L.orc_stream.argtypes = [C.c_int] * 3 + [_ip, _dp, _dp]
        L.orc_step.argtypes = [C.c_int] * 3 + [_ip, C.c_void_p, C.c_void_p, C.c_double, _dp, _dp, C.c_int]
        L.orc_run.argtypes = [C.c_int] * 3 + [_ip, C.c_void_p, C.c_void_p, C.c_double, C.c_int, _dp, _dp, C.c_int]
        L.orc_step_geom.argtypes = [C.c_int] * 3 + [_ip] + [C.c_void_p] * 5 + [C.c_double, _dp, _dp, C.c_int]
        L.orc_run_geom.argtypes = [C.c_int] * 3 + [_ip] + [C.c_void_p] * 5 + [C.c_double, C.c_int, _dp, _dp,
                                                                              C.c_int]
        L.orc_collide_force.argtypes = [_dp, C.c_double, _dp]
        L.orc_close_rule.argtypes = [C.c_int, _dp]
        L.orc_rule_unknowns.argtypes = [C.c_int, _ip]
        L.orc_check_geometry.argtypes = [C.c_int] * 3 + [_ip, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]
        L.orc_init_equilibrium.argtypes = [C.c_int] * 3 + [C.c_double, _dp]
        L.orc_macros.argtypes = [C.c_int] * 3 + [_dp, _dp, _dp]
        L.orc_reduce.argtypes = [C.c_int] * 3 + [_dp, C.c_void_p, _dp]
        L.orc_sources.argtypes = [C.c_int] * 3 + [_ip, C.c_int64, _lp, _lp]
        L.orc_update_gathered.argtypes = [C.c_int] * 3 + [_ip, C.c_void_p, C.c_void_p, C.c_double, C.c_int64,
                                                          _lp, _dp, _dp, C.c_int]
        L.orc_lattice.argtypes = [_ip, _dp, _ip]
        L.orc_threads.restype = C.c_int
        for name in ("orc_close_face", "orc_close_edge", "orc_close_corner", "orc_close_face_pressure", "orc_stream",
                     "orc_step", "orc_run", "orc_step_geom", "orc_run_geom", "orc_sources", "orc_update_gathered",
                     "orc_close_rule", "orc_rule_unknowns", "orc_check_geometry"):
            getattr(L, name).restype = C.c_int
        _LIB = L
    return _LIB


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def lattice():
    """(c[19,3] int, w[19], opp[19]) as tabulated in the oracle."""
    c = np.zeros(Q * 3, np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    lib().orc_lattice(c, w, opp)
    return c.reshape(Q, 3), w, opp


def feq(rho: float, u) -> np.ndarray:
    out = np.zeros(Q)
    lib().orc_feq(float(rho), np.ascontiguousarray(u, np.float64), out)
    return out


def moments(f) -> tuple[float, np.ndarray]:
    out = np.zeros(4)
    lib().orc_moments(np.ascontiguousarray(f, np.float64), out)
    return out[0], out[1:].copy()


def collide(f, tau: float) -> np.ndarray:
    g = np.array(f, np.float64)
    lib().orc_collide(g, float(tau))
    return g


def close_face(face: int, f, u, form: int = 0):
    """Face closure of one node; returns (closed populations, rho)."""
    g = np.array(f, np.float64)
    rho = C.c_double()
    _check(lib().orc_close_face(face, form, g, np.ascontiguousarray(u, np.float64), C.byref(rho)),
           "close_face")
    return g, rho.value


def close_face_pressure(face: int, f, rho0: float, u_t, form: int = 0):
    """Pressure closure of one node: density rho0 and tangential velocity u_t (normal
    component ignored) prescribed; returns (closed populations, normal velocity)."""
    g = np.array(f, np.float64)
    vn = C.c_double()
    _check(lib().orc_close_face_pressure(face, form, g, float(rho0), np.ascontiguousarray(u_t, np.float64),
                                         C.byref(vn)), "close_face_pressure")
    return g, vn.value


def collide_force(f, tau: float, force) -> np.ndarray:
    """BGK collision with the body force of eq. gravity (velocity shift tau F / rho)."""
    g = np.array(f, np.float64)
    lib().orc_collide_force(g, float(tau), np.ascontiguousarray(force, np.float64))
    return g


def close_rule(code: int, f) -> np.ndarray:
    """Boundary rule of a node code of a general geometry (no-slip)."""
    g = np.array(f, np.float64)
    _check(lib().orc_close_rule(int(code), g), "close_rule")
    return g


def rule_unknowns(code: int) -> np.ndarray:
    """Boolean mask of the populations the rule of ``code`` overwrites."""
    out = np.zeros(Q, np.int32)
    _check(lib().orc_rule_unknowns(int(code), out), "rule_unknowns")
    return out.astype(bool)


def check_geometry(lat: "Lattice") -> int:
    """-1 if the lattice's node codes are consistent with its solid nodes and walls,
    else the flat index of the first offending node."""
    bad = C.c_int64(0)
    rc = lib().orc_check_geometry(*lat.dims(), lat.kinds, lat._solid_ptr, lat._code_ptr, C.byref(bad))
    return -1 if rc == 0 else int(bad.value) - 1


def close_edge(face_a: int, face_b: int, f, rho_p: float = -1.0) -> np.ndarray:
    """No-slip edge; rho_p > 0 when the edge borders a pressure plane of that density."""
    g = np.array(f, np.float64)
    _check(lib().orc_close_edge(face_a, face_b, g, float(rho_p)), "close_edge")
    return g


def close_corner(face_x: int, face_y: int, face_z: int, f, rho_p: float = -1.0) -> np.ndarray:
    """No-slip corner; rho_p > 0 when the corner borders a pressure plane."""
    g = np.array(f, np.float64)
    _check(lib().orc_close_corner(face_x, face_y, face_z, g, float(rho_p)), "close_corner")
    return g


class Lattice:
    """A lattice description for the oracle: dims, face kinds and boundary tables.

    ``kinds[i]``: 0 periodic, 1 velocity, 2 pressure. ``utabs[i]`` is a float64 array of
    shape (n2, n1, 3) over the face's two tangential axes in increasing axis order (the
    prescribed velocity; for a pressure face its tangential part), or None for a
    periodic face. ``ptabs[i]`` is the (n2, n1) prescribed density of a pressure face.
    ``solid`` is an optional (nz, ny, nx) mask of solid nodes (mid-grid bounce-back).
    ``code`` is an optional (nz, ny, nx) int8 array of on-site boundary rules (see
    ``close_rule``); ``force`` the body force of eq. gravity.
    """

    def __init__(self, nx, ny, nz, kinds, utabs, tau, ptabs=None, solid=None, code=None, force=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.kinds = np.ascontiguousarray(kinds, np.int32)
        self.tau = float(tau)
        self._tabs = []
        ptrs = (C.c_void_p * 6)()
        pptrs = (C.c_void_p * 6)()
        ptabs = ptabs if ptabs is not None else [None] * 6
        for i in range(6):
            t = utabs[i]
            if t is None:
                t = np.zeros(3)
            t = np.ascontiguousarray(t, np.float64)
            self._tabs.append(t)
            ptrs[i] = t.ctypes.data
            if ptabs[i] is not None:
                pt = np.ascontiguousarray(ptabs[i], np.float64)
                self._tabs.append(pt)
                pptrs[i] = pt.ctypes.data
        self._ptrs = ptrs
        self._pptrs = pptrs
        self.solid = None if solid is None else np.ascontiguousarray(solid, np.uint8)
        if self.solid is not None and self.solid.shape != (self.nz, self.ny, self.nx):
            raise ValueError("solid mask must be (nz, ny, nx)")
        self.code = None if code is None else np.ascontiguousarray(code, np.int8)
        if self.code is not None and self.code.shape != (self.nz, self.ny, self.nx):
            raise ValueError("code array must be (nz, ny, nx)")
        self.force = None if force is None else np.ascontiguousarray(force, np.float64).reshape(3)

    @property
    def _solid_ptr(self):
        return None if self.solid is None else self.solid.ctypes.data

    @property
    def _code_ptr(self):
        return None if self.code is None else self.code.ctypes.data

    @property
    def _force_ptr(self):
        return None if self.force is None else self.force.ctypes.data

    @classmethod
    def from_workload(cls, wl):
        return cls(wl.nx, wl.ny, wl.nz, wl.kinds, wl.utabs, wl.tau, getattr(wl, "ptabs", None),
                   getattr(wl, "solid", None), getattr(wl, "code", None), getattr(wl, "force", None))

    @property
    def shape(self):
        return (Q, self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def dims(self):
        return self.nx, self.ny, self.nz


def init_equilibrium(lat: Lattice, rho0: float = 1.0) -> np.ndarray:
    f = np.zeros(lat.shape)
    lib().orc_init_equilibrium(*lat.dims(), float(rho0), f)
    return f


def stream(lat: Lattice, f) -> np.ndarray:
    fin = np.ascontiguousarray(f, np.float64)
    out = np.zeros(lat.shape)
    _check(lib().orc_stream(*lat.dims(), lat.kinds, fin, out), "stream")
    return out


# closure forms: 0 explicit per-plane formulas, 1 compact rule, 3 the compact rule with
# the transverse corrections forced to zero (the paper's N = 0 comparison closure)
FORM_EXPLICIT, FORM_COMPACT, FORM_COMPACT_NO_N = 0, 1, 3


def step(lat: Lattice, f, form: int = 0) -> np.ndarray:
    fin = np.ascontiguousarray(f, np.float64)
    out = np.zeros(lat.shape)
    _check(lib().orc_step_geom(*lat.dims(), lat.kinds, lat._ptrs, lat._pptrs, lat._solid_ptr, lat._code_ptr,
                               lat._force_ptr, lat.tau, fin, out, form), "step")
    return out


def run(lat: Lattice, f, nsteps: int, form: int = 0) -> np.ndarray:
    g = np.array(f, np.float64, order="C")
    work = np.empty_like(g)
    _check(lib().orc_run_geom(*lat.dims(), lat.kinds, lat._ptrs, lat._pptrs, lat._solid_ptr, lat._code_ptr,
                              lat._force_ptr, lat.tau, int(nsteps), g, work, form), "run")
    return g


def macros(lat: Lattice, f):
    """(rho[nz,ny,nx], u[3,nz,ny,nx]) of a stored state."""
    fin = np.ascontiguousarray(f, np.float64)
    rho = np.zeros(lat.shape[1:])
    u = np.zeros((3,) + lat.shape[1:])
    lib().orc_macros(*lat.dims(), fin, rho, u)
    return rho, u


def reduce(lat: Lattice, f, u_prev=None):
    """(sum rho, sum |u-u_prev|^2, sum |u|^2, bad-node count) in node order."""
    fin = np.ascontiguousarray(f, np.float64)
    out = np.zeros(4)
    up = None if u_prev is None else np.ascontiguousarray(u_prev, np.float64)
    lib().orc_reduce(*lat.dims(), fin, None if up is None else up.ctypes.data, out)
    return out


def residual(lat: Lattice, f, u_prev) -> float:
    _, du2, u2, _ = reduce(lat, f, u_prev)
    return float(np.sqrt(du2) / np.sqrt(u2)) if u2 > 0 else float(np.sqrt(du2))


def sources(lat: Lattice, nodes) -> np.ndarray:
    nodes = np.ascontiguousarray(nodes, np.int64)
    src = np.zeros((len(nodes), Q), np.int64)
    _check(lib().orc_sources(*lat.dims(), lat.kinds, len(nodes), nodes, src), "sources")
    return src


def update_gathered(lat: Lattice, nodes, gathered, form: int = 0) -> np.ndarray:
    nodes = np.ascontiguousarray(nodes, np.int64)
    g = np.ascontiguousarray(gathered, np.float64).reshape(len(nodes), Q)
    out = np.zeros_like(g)
    _check(lib().orc_update_gathered(*lat.dims(), lat.kinds, lat._ptrs, lat._pptrs, lat.tau, len(nodes),
                                     nodes, g, out, form), "update_gathered")
    return out


def threads() -> int:
    return int(lib().orc_threads())


def step_nodes(lat: Lattice, value_at, nodes, form: int = 0) -> np.ndarray:
    """One time step evaluated only at ``nodes``.

    ``value_at(flat_indices)`` returns the pre-step state at flat indices
    ``k*N + node``; only the pull sources of the listed nodes are requested, so a
    lattice far larger than host memory can be checked node by node.
    """
    src = sources(lat, nodes)
    g = np.full(src.shape, np.nan)
    known = src >= 0
    g[known] = value_at(src[known])
    return update_gathered(lat, nodes, g, form)

