"""GB300-native first-order immersed-boundary time step (Givelberg & Bunn, Section 3.2).

The compute path is the CUDA library ``libibgb.so`` (built from ``csrc/``)
behind the C ABI declared in ``include/ib.h``; ``binding`` is its thin ctypes
binding.  ``synth`` generates seeded synthetic inputs.  Importing this package
loads nothing; ``binding.load()`` loads the library and fails loudly if it is
missing.
"""
__all__ = ["synth", "binding"]
