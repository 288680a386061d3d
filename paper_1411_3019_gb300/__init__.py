"""surfmd: constrained Langevin molecular dynamics on implicit surfaces
(Paquay & Kusters, Algorithm 1 and Algorithm S1) on one GB300 GPU.

The compute path is the CUDA library ``libsurfmd.so`` built from ``csrc/``;
``md`` is its thin ctypes binding and ``inputs`` the seeded workload
generators. Importing the package loads nothing; ``md`` loads the library
on first use and raises if it is missing.
"""
__all__ = ["md", "inputs"]
