"""GB300-native (sm_103a) hot path of the 3D radiative transfer framework of
Hauschildt & Baron (2011): characteristics formal solution on an x/y
periodic slab, nearest-neighbour Lambda*, operator-splitting update of J and
the iteration to convergence.

``rt3d`` is the thin ctypes binding of the C-ABI library ``librt3d.so``;
``workloads`` draws the seeded synthetic slabs.  Importing this package
loads nothing; ``rt3d`` loads the CUDA library on first use and raises if it
is missing.
"""

__all__ = ["rt3d", "workloads"]
