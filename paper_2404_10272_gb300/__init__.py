"""GB300-native occupancy-grid ray sampler with VDB-style grids and
hierarchical DDA (Kato & Tarashima, CVPR-W 2024).

The compute path is the CUDA library ``libhdda`` (see ``include/hdda.h``);
``paper_2404_10272_gb300.hdda`` is its thin ctypes binding.  ``scenes`` holds
the seeded synthetic input generators.  Importing the package does not load
the CUDA library; the first call into ``hdda`` does, and fails loudly when it
is missing.
"""
__all__ = ["scenes", "hdda"]
