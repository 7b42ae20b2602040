"""GB300-native SPH neighbour-interaction hot path (cell binning, density with the
smoothing-length iteration, pressure force with artificial viscosity, KDK step)
after Theuns et al. 2015, "Swift: task-based hydrodynamics and gravity for
cosmological simulations", Sec. 2 and Sec. 3.1.

The compute lives in hand-written CUDA kernels behind the C-ABI library
``libsph.so`` (declared in ``include/sph.h``); :mod:`.binding` marshals
arguments only.  Importing this package does not load the library; call
:func:`paper_1508_00115_gb300.binding.lib` (or build it with
:func:`paper_1508_00115_gb300.build.build`).
"""
__all__ = ["binding", "build", "inputs"]
