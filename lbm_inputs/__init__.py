"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no lattice-Boltzmann arithmetic. It only defines
  * a counter-based random generator (SplitMix64, Steele, Lea & Flood, OOPSLA 2014),
  * the lattice sizes, relaxation times and face kinds of each workload,
  * the prescribed boundary-velocity tables of each workload (uniform vectors and
    parabolic profiles evaluated at node positions),
  * the request stream of the serving workload.

Face numbering: 0: x=0, 1: x=nx-1, 2: y=0, 3: y=ny-1, 4: z=0, 5: z=nz-1. A velocity
face carries a float64 table of shape (n2, n1, 3) over its two tangential axes in
increasing axis order (x faces: [z][y], y faces: [z][x], z faces: [y][x]); a pressure
face carries a density table (n2, n1) and a velocity table whose tangential part is the
prescribed tangential velocity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC = 0
VELOCITY = 1
PRESSURE = 2

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser of a uint64 counter array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, np.uint64) + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform [0, 1) doubles at counter positions ``idx`` of (seed, stream)."""
    idx = np.asarray(idx, np.uint64)
    with np.errstate(over="ignore"):
        key = splitmix64(np.uint64(seed) * np.uint64(0x100000001B3) + np.uint64(stream))
        bits = splitmix64(idx ^ key)
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def face_shape(face: int, nx: int, ny: int, nz: int) -> tuple[int, int]:
    """(n2, n1) of the velocity table of a face."""
    dims = (nx, ny, nz)
    a = face // 2
    t1, t2 = [b for b in range(3) if b != a]
    return dims[t2], dims[t1]


def uniform_table(face: int, nx: int, ny: int, nz: int, u) -> np.ndarray:
    n2, n1 = face_shape(face, nx, ny, nz)
    t = np.empty((n2, n1, 3))
    t[...] = np.asarray(u, np.float64)
    return t


def parabola(n: int) -> np.ndarray:
    """Profile 4 s (n-1-s) / (n-1)^2 on nodes s = 0..n-1: 0 on both end nodes, 1 at
    the centre of an odd count."""
    s = np.arange(n, dtype=np.float64)
    return 4.0 * s * (n - 1 - s) / float((n - 1) ** 2)


@dataclass
class Workload:
    """One lattice solve: sizes, relaxation time, face kinds and velocity tables."""
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    kinds: tuple
    utabs: list
    rho0: float = 1.0
    steps: int = 0
    meta: dict = field(default_factory=dict)
    ptabs: list = field(default_factory=lambda: [None] * 6)
    solid: object = None  # optional (nz, ny, nx) uint8 mask of solid nodes
    code: object = None   # optional (nz, ny, nx) int8 on-site boundary rule codes
    force: object = None  # optional body force (3,)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dims(self):
        return self.nx, self.ny, self.nz


def make_workload(name, nx, ny, nz, tau, face_u, steps=0, rho0=1.0, meta=None, face_p=None) -> Workload:
    """``face_u[i]`` is None (periodic), a 3-vector (uniform) or a (n2, n1, 3) table;
    ``face_p[i]``, when given, makes face i a pressure face with that density (a scalar
    or an (n2, n1) table) and face_u[i] its tangential velocity (zero if None)."""
    face_p = face_p or [None] * 6
    kinds, tabs, ptabs = [], [], []
    for i in range(6):
        fu, fp = face_u[i], face_p[i]
        if fu is None and fp is None:
            kinds.append(PERIODIC)
            tabs.append(None)
            ptabs.append(None)
            continue
        kinds.append(PRESSURE if fp is not None else VELOCITY)
        arr = np.asarray(fu if fu is not None else ZERO, np.float64)
        if arr.shape == (3,):
            arr = uniform_table(i, nx, ny, nz, arr)
        if arr.shape != face_shape(i, nx, ny, nz) + (3,):
            raise ValueError(f"face {i}: table shape {arr.shape}")
        tabs.append(np.ascontiguousarray(arr))
        if fp is None:
            ptabs.append(None)
        else:
            pt = np.empty(face_shape(i, nx, ny, nz))
            pt[...] = np.asarray(fp, np.float64)
            ptabs.append(pt)
    return Workload(name, nx, ny, nz, tau, tuple(kinds), tabs, rho0, steps, meta or {}, ptabs)


ZERO = (0.0, 0.0, 0.0)


def couette(nx=8, ny=8, nz=17, tau=1.0, u_top=0.05, steps=5000) -> Workload:
    """Shear flow: x, y periodic; wall at z=0 at rest, wall at z=nz-1 moving with
    (u_top, 0, 0)."""
    return make_workload("couette", nx, ny, nz, tau,
                         [None, None, None, None, ZERO, (u_top, 0.0, 0.0)], steps,
                         meta={"u_top": u_top})


def shear(nx=32, ny=32, nz=32, tau=1.0, u=0.02, steps=0) -> Workload:
    """The paper's shear test: x, y periodic; the bottom plane z=0 moves with (-u, 0, 0)
    and the top plane z=nz-1 with (+u, 0, 0)."""
    return make_workload("shear", nx, ny, nz, tau, [None, None, None, None, (-u, 0.0, 0.0), (u, 0.0, 0.0)],
                         steps, meta={"u": u})


def duct(nx=256, ny=64, nz=64, tau=0.6, peak=0.05, angle_deg=30.0, steps=20000) -> Workload:
    """Square duct: velocity inlet at x=0 with a product-parabola profile of the given
    peak, tilted by ``angle_deg`` from the x axis in the x-y plane; the same profile
    prescribed at the outlet x=nx-1; resting walls on the y and z faces."""
    a = math.radians(angle_deg)
    prof = peak * np.outer(parabola(nz), parabola(ny))            # [z][y]
    tab = np.stack([prof * math.cos(a), prof * math.sin(a), np.zeros_like(prof)], axis=-1)
    return make_workload("duct", nx, ny, nz, tau, [tab, tab, ZERO, ZERO, ZERO, ZERO], steps,
                         meta={"peak": peak, "angle_deg": angle_deg})


def channel(nx=512, ny=512, nz=512, tau=0.8, u=(0.04, 0.01, 0.0), steps=1000) -> Workload:
    """Channel: uniform velocity u at the inlet x=0 and the outlet x=nx-1, periodic in
    y, resting walls at z=0 and z=nz-1."""
    return make_workload("channel", nx, ny, nz, tau, [u, u, None, None, ZERO, ZERO], steps,
                         meta={"u": tuple(u)})


def poiseuille(lz=32, tau=1.0, peak=0.02, lx=4, ly=4, steps=0) -> Workload:
    """Plane channel between resting walls at z=0 and z=lz-1, periodic in y, with the
    parabolic profile peak*phi(z) x-hat prescribed at the inlet x=0 and outlet x=lx-1."""
    prof = peak * np.repeat(parabola(lz)[:, None], ly, axis=1)   # [z][y]
    tab = np.stack([prof, np.zeros_like(prof), np.zeros_like(prof)], axis=-1)
    return make_workload("poiseuille", lx, ly, lz, tau, [tab, tab, None, None, ZERO, ZERO], steps,
                         meta={"peak": peak})


def pressure_duct(n=16, length=48, tau=1.0, rho_in=1.005, rho_out=0.995, steps=0) -> Workload:
    """Pressure-driven square duct: n x n cross-section with resting walls on the y and
    z faces (walls on the end nodes, width n-1), density rho_in at x=0 and rho_out at
    x=length-1, no tangential velocity on the pressure planes."""
    return make_workload("pressure_duct", length, n, n, tau, [None, None, ZERO, ZERO, ZERO, ZERO], steps,
                         meta={"rho_in": rho_in, "rho_out": rho_out},
                         face_p=[rho_in, rho_out, None, None, None, None])


def tilted_channel(scale: int = 1, tau: float = 1.0, u0: float = 0.01, shift: int = 40, normal_only=False,
                   steps: int = 20000) -> Workload:
    """The tilted-channel geometry of the paper's numerical results: a 64 x 8 x 128
    domain (times ``scale``), periodic in x and y; a channel 20 nodes wide along x whose
    centre line moves by ``shift`` nodes in x over the 127 node spacings in z (zero:
    the straight channel); solid nodes outside it; the Poiseuille profile along the
    channel axis prescribed on the fluid nodes of the planes z = 0 and z = nz - 1.

    Fluid nodes satisfy |x - x_c(z)| < w/2 with x_c(z) = x0 + g (z - z0), (x0, z0) the
    centre of the domain, g = shift / 127, w = 20 (all lengths times ``scale``). The
    profile is v(x) = u0 [1 - ((x - x_c(z)) / (w/2))^2] along (g, 0, 1) / |(g, 0, 1)|
    (eq. pois). ``normal_only`` gives the comparison inflow restricted to the plane
    normal: True (or "component") keeps the profile's z component, "magnitude" puts its
    full speed along z."""
    nx, ny, nz = 64 * scale, 8 * scale, 128 * scale
    g = shift / 127.0
    half = 10.0 * scale
    x0, z0 = (nx - 1) / 2.0, (nz - 1) / 2.0
    x = np.arange(nx)[None, None, :]
    z = np.arange(nz)[:, None, None]
    d = (x - x0 - g * (z - z0)) / half + 0.0 * np.zeros((1, ny, 1))
    solid = (np.abs(d) >= 1.0).astype(np.uint8)
    direction = np.array([g, 0.0, 1.0]) / math.hypot(g, 1.0)
    prof = np.where(solid == 0, u0 * (1.0 - d * d), 0.0)          # [z][y][x]
    vel = prof[..., None] * direction                               # [z][y][x][3]
    if normal_only not in (False, True, "component", "magnitude"):
        raise ValueError("normal_only must be False, True, 'component' or 'magnitude'")
    if normal_only == "magnitude":
        vel[..., 2] = prof
    if normal_only:
        vel[..., 0] = 0.0
        vel[..., 1] = 0.0
    # z faces: tables [y][x][3]
    bottom = np.ascontiguousarray(vel[0])
    top = np.ascontiguousarray(vel[-1])
    wl = make_workload("tilted_channel", nx, ny, nz, tau, [None, None, None, None, bottom, top], steps,
                       meta={"u0": u0, "gamma": g, "half_width": half, "x0": x0, "z0": z0, "scale": scale,
                             "direction": direction.tolist(), "normal_only": normal_only})
    wl.solid = np.ascontiguousarray(solid)
    return wl


# ------------------------------------------------------------------------------------
# General geometries: per-node boundary codes (the normal stored on the node as a
# lattice-vector index, as the C ABI defines them) and body forces.
# ------------------------------------------------------------------------------------

# The paper's lattice vectors c_1..c_18 (columns of its matrix M); a code names a
# normal by its index here.
PAPER_VECTORS = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                 (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (-1, 1, 0), (-1, -1, 0),
                 (-1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1))


def vector_index(v) -> int:
    """Paper index (1..18) of a lattice vector."""
    return PAPER_VECTORS.index(tuple(int(a) for a in v)) + 1


def plane_code(n) -> int:
    return vector_index(n)


def concave_edge_code(n1, n2) -> int:
    return vector_index(np.add(n1, n2))


def convex_edge_code(n1, n2) -> int:
    return -vector_index(np.add(n1, n2))


def corner_code(n) -> int:
    sx, sy, sz = (int(a) for a in n)
    return 19 + (sx < 0) + 2 * (sy < 0) + 4 * (sz < 0)


def junction_code(n_plane, n1, n2) -> int:
    """Convex edge with plane normals n1, n2 meeting the plane with normal n_plane."""
    p = vector_index(n_plane)
    d = tuple(int(a) for a in np.add(n1, n2))
    perp = [v for v in PAPER_VECTORS[6:] if sum(a * b for a, b in zip(v, n_plane)) == 0]
    return 27 + 4 * (p - 1) + perp.index(d)


def _axis_vec(a: int, s: int):
    v = [0, 0, 0]
    v[a] = s
    return v


def force_poiseuille(n: int = 32, tau: float = 2.0, force: float = 1e-5, wall_axis: int = 0, flow_axis: int = 2,
                     other: int = 3, steps: int = 0) -> Workload:
    """Plane Poiseuille flow driven by a body force (the paper's 32^3 check): resting
    walls on both faces of ``wall_axis`` (n nodes, walls on the end nodes), periodic
    on the other axes (``other`` nodes each, except ``n`` on the flow axis when other
    is None), force along ``flow_axis``."""
    dims = [other if other is not None else n] * 3
    dims[wall_axis] = n
    face_u = [None] * 6
    face_u[2 * wall_axis] = ZERO
    face_u[2 * wall_axis + 1] = ZERO
    wl = make_workload("force_poiseuille", dims[0], dims[1], dims[2], tau, face_u, steps,
                       meta={"wall_axis": wall_axis, "flow_axis": flow_axis, "force": force})
    f = np.zeros(3)
    f[flow_axis] = force
    wl.force = f
    return wl


def embedded_walls(wl: Workload) -> Workload:
    """The same lattice with its walled faces moved inside the domain: one layer of
    solid nodes is added beyond every walled face, and the former boundary nodes carry
    the codes of the planes, concave edges and corners they lie on. All walls of ``wl``
    must be at rest (no-slip)."""
    nx, ny, nz = wl.dims
    walled = [wl.kinds[2 * a] != PERIODIC for a in range(3)]
    for i in range(6):
        if wl.kinds[i] == PRESSURE or (wl.kinds[i] == VELOCITY and np.any(wl.utabs[i] != 0.0)):
            raise ValueError("embedded_walls needs resting walls")
    pad = [1 if w else 0 for w in walled]
    dims = [n + 2 * p for n, p in zip((nx, ny, nz), pad)]
    solid = np.ones((dims[2], dims[1], dims[0]), np.uint8)
    solid[pad[2]:pad[2] + nz, pad[1]:pad[1] + ny, pad[0]:pad[0] + nx] = 0
    code = np.zeros_like(solid, dtype=np.int8)
    size = (nx, ny, nz)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = (x, y, z)
                normals = []
                for a in range(3):
                    if not walled[a]:
                        continue
                    if c[a] == 0:
                        normals.append(_axis_vec(a, 1))
                    elif c[a] == size[a] - 1:
                        normals.append(_axis_vec(a, -1))
                if not normals:
                    continue
                if len(normals) == 1:
                    k = plane_code(normals[0])
                elif len(normals) == 2:
                    k = concave_edge_code(*normals)
                else:
                    k = corner_code(np.sum(normals, axis=0))
                code[z + pad[2], y + pad[1], x + pad[0]] = k
    face_u = [None if not walled[i // 2] else ZERO for i in range(6)]
    out = make_workload(wl.name + "_embedded", dims[0], dims[1], dims[2], wl.tau, face_u, wl.steps, wl.rho0,
                        dict(wl.meta, pad=pad))
    out.solid = solid
    out.code = code
    out.force = None if wl.force is None else np.array(wl.force, np.float64)
    return out


def pillar_channel(n=(24, 16, 12), axis: int = 2, flow: int = 0, block=((9, 14), (5, 10)), tau: float = 0.9,
                   force: float = 2e-6) -> Workload:
    """A rectangular pillar spanning a channel between two resting walls, driven by a
    body force. ``axis`` is the pillar axis (its two faces are the walls), ``flow``
    the force direction (perpendicular to ``axis``); the other two axes are periodic.
    ``block`` gives the pillar's extent [lo, hi] (surface nodes included) on the two
    axes other than ``axis``, in increasing axis order. The pillar's surface nodes are
    boundary nodes with codes (planes, convex edges along the pillar, concave edges
    and edge/plane junctions where it meets the walls); its interior is solid. ``n``
    holds (n along axis, n along the first other axis, n along the second)."""
    others = [a for a in range(3) if a != axis]
    if flow not in others:
        raise ValueError("the force must be perpendicular to the pillar")
    dims = [0, 0, 0]
    dims[axis] = n[2]
    dims[others[0]] = n[0]
    dims[others[1]] = n[1]
    nx, ny, nz = dims
    solid = np.zeros((nz, ny, nx), np.uint8)
    code = np.zeros((nz, ny, nx), np.int8)
    (l0, h0), (l1, h1) = block
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = (x, y, z)
                u, v, w = c[others[0]], c[others[1]], c[axis]
                if not (l0 <= u <= h0 and l1 <= v <= h1):
                    continue
                if l0 < u < h0 and l1 < v < h1:
                    solid[z, y, x] = 1
                    continue
                # surface node: bulk-side normals of the pillar faces it lies on
                pn = []
                if u == l0:
                    pn.append(_axis_vec(others[0], -1))
                if u == h0:
                    pn.append(_axis_vec(others[0], 1))
                if v == l1:
                    pn.append(_axis_vec(others[1], -1))
                if v == h1:
                    pn.append(_axis_vec(others[1], 1))
                wall = None
                if w == 0:
                    wall = _axis_vec(axis, 1)
                elif w == dims[axis] - 1:
                    wall = _axis_vec(axis, -1)
                if len(pn) == 1:
                    k = plane_code(pn[0]) if wall is None else concave_edge_code(pn[0], wall)
                else:
                    k = convex_edge_code(pn[0], pn[1]) if wall is None else junction_code(wall, pn[0], pn[1])
                code[z, y, x] = k
    face_u = [None] * 6
    face_u[2 * axis] = ZERO
    face_u[2 * axis + 1] = ZERO
    wl = make_workload("pillar_channel", nx, ny, nz, tau, face_u,
                       meta={"axis": axis, "flow": flow, "block": block, "force": force})
    f = np.zeros(3)
    f[flow] = force
    wl.solid = solid
    wl.code = code
    wl.force = f
    return wl


def random_pressure_workload(seed: int, nx: int, ny: int, nz: int, tau: float, periodic_y: bool = False,
                             amp: float = 0.02) -> Workload:
    """Pressure faces at x=0 and x=nx-1 with random densities 1 +- amp and random
    tangential velocities; random velocity tables on the y and z faces (y periodic on
    request)."""
    face_u, face_p = [], []
    for i in range(6):
        if i in (2, 3) and periodic_y:
            face_u.append(None)
            face_p.append(None)
            continue
        n2, n1 = face_shape(i, nx, ny, nz)
        r = uniform(seed, 200 + i, np.arange(n2 * n1 * 3)).reshape(n2, n1, 3)
        face_u.append(0.04 * (2.0 * r - 1.0))
        if i < 2:
            q = uniform(seed, 210 + i, np.arange(n2 * n1)).reshape(n2, n1)
            face_p.append(1.0 + amp * (2.0 * q - 1.0))
        else:
            face_p.append(None)
    return make_workload(f"random_pressure{seed}", nx, ny, nz, tau, face_u, face_p=face_p)


def random_face_workload(seed: int, nx: int, ny: int, nz: int, tau: float, periodic=(False, False, False),
                         amp: float = 0.05) -> Workload:
    """Random velocity tables on every walled face (for boundary-rule checks)."""
    face_u = []
    for i in range(6):
        if periodic[i // 2]:
            face_u.append(None)
            continue
        n2, n1 = face_shape(i, nx, ny, nz)
        r = uniform(seed, 100 + i, np.arange(n2 * n1 * 3)).reshape(n2, n1, 3)
        face_u.append(amp * (2.0 * r - 1.0))
    return make_workload(f"random{seed}", nx, ny, nz, tau, face_u)


# ------------------------------------------------------------------------------------
# Random perturbation fields for non-equilibrium test states.
# ------------------------------------------------------------------------------------

def noise(seed: int, shape, stream: int = 0) -> np.ndarray:
    """Uniform [-1, 1) doubles of a given shape (counter = flat index)."""
    n = int(np.prod(shape))
    return (2.0 * uniform(seed, stream, np.arange(n, dtype=np.uint64)) - 1.0).reshape(shape)


def noise_at(seed: int, shape, flat_idx, stream: int = 0) -> np.ndarray:
    """Values of ``noise(seed, shape, stream)`` at flat indices, without building it."""
    del shape
    return 2.0 * uniform(seed, stream, np.asarray(flat_idx, np.uint64)) - 1.0


def separable_noise_tables(seed: int, nx: int, ny: int, nz: int, q: int = 19, period: int = 61):
    """Small random tables whose broadcast sum gives a cheap large-lattice field:
    eps[k,z,y,x] = (a[k,x] + b[k,y] + c[k,z] + d[k,(7x+13y+29z) mod period]) / 4."""
    a = noise(seed, (q, nx), 1)
    b = noise(seed, (q, ny), 2)
    c = noise(seed, (q, nz), 3)
    d = noise(seed, (q, period), 4)
    return a, b, c, d


def separable_noise_at(tables, nx: int, ny: int, nz: int, flat_idx, q: int = 19, period: int = 61):
    a, b, c, d = tables
    flat_idx = np.asarray(flat_idx, np.int64)
    n = nx * ny * nz
    k = flat_idx // n
    node = flat_idx % n
    x = node % nx
    y = (node // nx) % ny
    z = node // (nx * ny)
    h = (7 * x + 13 * y + 29 * z) % period
    return (a[k, x] + b[k, y] + c[k, z] + d[k, h]) / 4.0


def separable_noise_slab(tables, nx: int, ny: int, z0: int, z1: int, q: int = 19, period: int = 61,
                         dtype=np.float64) -> np.ndarray:
    """The field for planes z0..z1-1 as an array (q, z1-z0, ny, nx)."""
    a, b, c, d = tables
    zs = np.arange(z0, z1)
    ys = np.arange(ny)
    xs = np.arange(nx)
    h = (7 * xs[None, None, :] + 13 * ys[None, :, None] + 29 * zs[:, None, None]) % period
    out = (a[:, None, None, :] + b[:, None, :, None] + c[:, zs][:, :, None, None] + d[:, h]) / 4.0
    return out.astype(dtype, copy=False)


# ------------------------------------------------------------------------------------
# Serving workload: a seeded stream of duct / channel solves.
# ------------------------------------------------------------------------------------

@dataclass
class Request:
    rid: int
    arrival_s: float
    kind: str
    nx: int
    ny: int
    nz: int
    speed: float
    angle_deg: float
    tau: float

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def serving_requests(n: int, seed: int, rate_hz: float, dmin: int = 32, dmax: int = 192):
    """n requests with Poisson arrivals at ``rate_hz``; dims log-uniform on
    [dmin, dmax] per axis; speed U(0.01, 0.08); direction angle U(0, 45) degrees in
    the x-y plane; tau U(0.55, 1.5); kind duct or channel with equal odds."""
    k = np.arange(n, dtype=np.uint64)
    u = [uniform(seed, 1000 + j, k) for j in range(8)]
    gaps = -np.log1p(-u[0]) / rate_hz
    t = np.cumsum(gaps)
    lo, hi = math.log(dmin), math.log(dmax)
    dims = [np.floor(np.exp(lo + (hi - lo) * u[1 + j])).astype(int) for j in range(3)]
    out = []
    for i in range(n):
        out.append(Request(i, float(t[i]), "duct" if u[4][i] < 0.5 else "channel",
                           int(dims[0][i]), int(dims[1][i]), int(dims[2][i]),
                           0.01 + 0.07 * float(u[5][i]), 45.0 * float(u[6][i]),
                           0.55 + 0.95 * float(u[7][i])))
    return out


def request_workload(r: Request) -> Workload:
    """The lattice solve a serving request asks for."""
    if r.kind == "duct":
        return duct(r.nx, r.ny, r.nz, r.tau, r.speed, r.angle_deg, steps=0)
    a = math.radians(r.angle_deg)
    return channel(r.nx, r.ny, r.nz, r.tau, (r.speed * math.cos(a), r.speed * math.sin(a), 0.0), steps=0)
