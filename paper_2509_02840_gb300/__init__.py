"""GB300-native Givens bidiagonal update (BGU) library.

The compute path is the C-ABI shared library built from ``csrc/`` (declared in
``include/bdu.h``); ``bdu`` is its thin ctypes binding.  ``inputs`` holds the
seeded synthetic workload generators shared by tests and benchmarks.
"""
__all__ = ["bdu", "inputs", "build"]


def __getattr__(name):
    if name in ("bdu", "inputs", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
