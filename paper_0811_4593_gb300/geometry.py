"""Boundary codes for a voxel geometry.

The on-site rules of complex geometries (Sec. "On-site no-slip boundary condition")
need every boundary node to carry its normal as an integer code (include/lbm.h,
``lbm_set_geometry``); the paper leaves finding them to the lattice generator. This
module derives them from a solid mask: a fluid node with at least one solid neighbour
gets the rule that overwrites every population it cannot stream (the source is solid or
lies outside a walled axis) and as few others as possible. The rule sets come from the
library itself (``lbm_rule_unknowns``), so the host needs no device.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._binding import LBMError, check, lib

CODES = tuple(range(1, 51)) + tuple(range(-18, -6))

# lattice vectors c_1..c_19 (the paper's matrix M), population k = c_{k+1}
_C = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
               (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (-1, 1, 0), (-1, -1, 0),
               (-1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1),
               (0, 0, 0)])


def rule_unknowns(code: int) -> int:
    """Bit mask of the populations the rule of ``code`` overwrites."""
    m = C.c_uint32()
    check(lib().lbm_rule_unknowns(int(code), C.byref(m)))
    return int(m.value)


def _rule_table():
    masks = np.array([rule_unknowns(c) for c in CODES], np.uint32)
    sizes = np.array([bin(int(m)).count("1") for m in masks])
    return masks, sizes


def blocked_masks(solid, walled=(True, True, True)):
    """Per node: bit k set when population k cannot be streamed (its pull source x - c_k
    is solid, or outside the domain on a walled axis), and bit 31 when only the domain
    walls block it (no solid source). ``solid`` is (nz, ny, nx); ``walled[a]`` False
    makes axis a periodic."""
    s = np.asarray(solid, bool)
    nz, ny, nx = s.shape
    out = np.zeros(s.shape, np.uint32)
    from_solid = np.zeros(s.shape, bool)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dims = (nx, ny, nz)
    for k in range(18):
        c = _C[k]
        src = [x - c[0], y - c[1], z - c[2]]
        outside = np.zeros(s.shape, bool)
        for a in range(3):
            if walled[a]:
                outside |= (src[a] < 0) | (src[a] >= dims[a])
            src[a] = np.mod(src[a], dims[a])
        solid_src = s[src[2], src[1], src[0]] & ~outside
        out |= np.where(outside | solid_src, np.uint32(1 << k), np.uint32(0))
        from_solid |= solid_src
    out |= np.where(from_solid, np.uint32(0), np.uint32(1 << 31))
    return out


def classify(solid, walled=(True, True, True), on_missing: str = "bounce_back") -> np.ndarray:
    """int8 codes (nz, ny, nx) for ``lbm_set_geometry``: 0 for solid nodes, for fluid
    nodes without a solid neighbour (bulk, or faces / edges / corners of the box, which
    the sweep classifies itself) and a rule code for every other fluid node.

    Where no rule of the paper covers a node's blocked populations, or two smallest rules
    tie (a fluid node between two solid nodes on one axis; the convex corner of a
    staircase, whose three blocked diagonals three junction rules would fit equally),
    the node keeps code 0 and the sweep applies mid-grid bounce-back to its links to
    solid nodes (``on_missing="bounce_back"``), or LBMError is raised
    (``on_missing="raise"``)."""
    if on_missing not in ("bounce_back", "raise"):
        raise ValueError("on_missing must be 'bounce_back' or 'raise'")
    s = np.asarray(solid, bool)
    blocked = blocked_masks(s, walled)
    codes = np.zeros(s.shape, np.int8)
    masks, sizes = _rule_table()
    need = (~s) & ((blocked & np.uint32(1 << 31)) == 0)
    for b in np.unique(blocked[need]):
        fits = (masks & b) == b
        choice = np.flatnonzero(fits & (sizes == sizes[fits].min())) if fits.any() else np.array([], int)
        if len(choice) != 1:
            if on_missing == "raise":
                z, y, x = np.argwhere(need & (blocked == b))[0]
                what = "no boundary rule sets all of its unstreamable populations" if len(choice) == 0 else \
                    f"rules {[CODES[i] for i in choice]} fit equally"
                raise LBMError(-1, f"node ({x}, {y}, {z}): {what} (mask {int(b):#07x})")
            continue
        codes[need & (blocked == b)] = CODES[choice[0]]
    return codes
