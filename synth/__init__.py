"""Seeded synthetic inputs (meshes, materials, transducer layouts, vectors).

This package holds no arithmetic of the boundary element method: it only
produces the plain arrays that both the CUDA library and the FP64 oracle take
as inputs.
"""
from . import meshes, scenes  # noqa: F401
