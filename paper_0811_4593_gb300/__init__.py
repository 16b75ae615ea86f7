"""GB300-native D3Q19 lattice Boltzmann solver with the on-site velocity boundary
condition of Hecht & Harting (arXiv:0811.4593).

The solver is the CUDA library ``liblbm.so`` (C ABI: include/lbm.h); this package is
its Python binding. Build it with ``paper_0811_4593_gb300.build.build()``.
"""
from . import geometry
from ._binding import (Batch, LBMDiverged, LBMError, Lattice, Pressure, lib, library_path,
                       use_default_allocator, use_torch_allocator)

__all__ = ["Lattice", "Batch", "Pressure", "LBMError", "LBMDiverged", "lib", "library_path", "use_torch_allocator",
           "use_default_allocator", "geometry"]
