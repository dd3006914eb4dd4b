"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only produces inputs: surface meshes (vertex coordinates and
oriented triangles) and seeded random complex vectors.  It holds none of the
solver's arithmetic (no basis functions, no Green's function, no grid), so the
oracle and the CUDA path can both consume its output without sharing any of
the method.
"""
from .meshes import icosphere, box, bar_cluster, mesh_edges_count
from .vectors import cn_vector

__all__ = ["icosphere", "box", "bar_cluster", "mesh_edges_count", "cn_vector"]
