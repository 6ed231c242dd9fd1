"""SACRA-2D hot path on one GB300 (sm_103a): one Runge-Kutta stage of
Z4c + HLLC GRHD on the fixed-mesh-refinement cartoon grid, as hand-written
CUDA kernels behind a C ABI (``include/sacra2d.h``).

The compiled library is loaded lazily by :mod:`paper_2502_03223_gb300.sacra2d`;
importing the package itself loads nothing.
"""
