"""GB300-native short-ranged Lennard-Jones MD over cell lists.

A CUDA library (``liblj.so``, C ABI declared in ``include/lj.h``) computes the
hot path of van Meel et al., arXiv:0709.3225, Section 3: per-step binning of
particles into cells, the periodic Lennard-Jones force over the 27
neighbouring cells, and the velocity-Verlet update.  ``paper_0709_3225_gb300.lj``
is the thin ctypes binding with the same entry-point names; ``inputs`` makes
the seeded synthetic workloads.

Importing this package loads nothing; the library is loaded on first use and
the binding raises if it has not been built.
"""
__all__ = ["inputs", "lj"]
