"""GB300-native solver for the 3D Eikonal equation |grad u| F = 1 by the
parallel Heap-Cell Method (Chacon & Vladimirsky, arXiv:1306.4743).

The compute path is the CUDA library ``libeik.so`` (csrc/), reached through
the C ABI declared in include/eik.h; ``eik`` is its Python binding and
``workloads`` holds the seeded synthetic inputs.  Submodules load lazily so
that importing the input generators never needs a GPU.
"""
__all__ = ["eik", "workloads"]
