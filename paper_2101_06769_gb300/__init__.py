"""GB300 (sm_103a) implementation of the multiphase lattice Boltzmann step of
Hosseini, Safari & Thevenin (arXiv 2101.06769): conservative Allen-Cahn
phase field + pressure-based cumulant flow solver, as a C-ABI CUDA library
with a thin ctypes binding."""
from .lbmp import (BF16_SHIFTED, Batch, CASE, D2Q9, D3Q27, EXPORTS, FLAG_DYNAMIC_VISC, FLAG_PHASE_REDUCED, FLAG_UNIFORM_FORCE,
                   FLAG_WE_LIGHT, FP16_SHIFTED, FP32, LIB_PATH, Domain, LbmpError, load, make_params)

__all__ = ["Domain", "Batch", "LbmpError", "load", "make_params", "CASE", "D2Q9", "D3Q27", "FP32", "FP16_SHIFTED",
           "BF16_SHIFTED", "FLAG_WE_LIGHT", "FLAG_DYNAMIC_VISC", "FLAG_UNIFORM_FORCE", "FLAG_PHASE_REDUCED", "EXPORTS",
           "LIB_PATH"]
