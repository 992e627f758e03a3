"""GB300-native non-nested geometric multigrid with the global-local combined smoother.

The compute path lives in the shared library built from ``csrc/`` (C++ host setup and
sm_103a CUDA kernels behind a C ABI declared in ``include/nnmg.h``); ``nnmg`` is the thin
ctypes binding over it. ``inputs`` holds the seeded synthetic meshes and right-hand sides.
Submodules are imported lazily so that importing the input generators never loads the
CUDA library.
"""

__all__ = ["inputs", "nnmg", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
