"""GB300-native implicit finite-element seismic wave analysis (arXiv 2404.17754).

The GPU library (``libgsw.so``, C ABI in ``include/gsw.h``) runs the
per-candidate 3D wave-propagation analysis; :mod:`.gsw` is its Python
binding.  Importing this package does not load the library; build it with
:func:`paper_2404_17754_gb300.build.build`.
"""
__all__ = ["build", "gsw"]
