"""B300-native discrete-ordinates (S_N) photon-transport solver.

The hot path -- multigroup source iteration with diamond-difference wavefront
sweeps, Legendre-moment scatter source and the Eq. 3 quadrature reduction of
the DOCTORS method (arxiv 1910.11335) -- runs in libdts.so (hand-written CUDA
for sm_103a) behind the C ABI of include/dts.h. ``dts`` is its Python binding
and ``inputs`` the seeded synthetic workload generators.
"""
__all__ = ["dts", "inputs"]
