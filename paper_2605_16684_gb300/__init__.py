"""GB300-native entropy-stable DG Euler + buoyancy hot path.

The compute path is libesdg.so (hand-written CUDA for sm_103a) behind the C ABI
of include/es_dg.h; this package holds its ctypes binding (``_lib``), the build
step (``_build``) and the seeded synthetic input generators (``inputs``).
"""
from . import inputs  # noqa: F401


def __getattr__(name):
    # the binding is imported lazily so that CPU-only users of ``inputs`` never
    # touch CUDA
    if name in ("Solver", "load", "EsDgError"):
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)
