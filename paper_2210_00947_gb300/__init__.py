"""GB300 (sm_103a) implementation of multigrid-assisted reanalysis (MGAR)
heat-transfer topology optimisation (Yin, Wang, Guo, Li, arXiv 2210.00947).

  workloads  seeded synthetic inputs (grids, heat-sink masks, loads, densities)
  mgar       Python binding of the C ABI in include/mgar.h (libmgar.so)
  build      in-tree nvcc build of libmgar.so for sm_103a

Importing the package loads nothing; the CUDA library is loaded on first use
of paper_2210_00947_gb300.mgar.
"""
__all__ = ["workloads", "mgar", "build"]
