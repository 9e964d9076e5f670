"""GPU concurrency-control engine for batched OLTP transactions on sm_103a.

The compute path is the C-ABI library built from ``csrc/`` (declared in
``include/gcc_gb300.h``); ``engine`` is its thin ctypes binding and
``workload`` holds the seeded synthetic input generators.  Submodules are
imported lazily so that the generators can be used without loading the
CUDA library.
"""
__all__ = ["engine", "workload"]
