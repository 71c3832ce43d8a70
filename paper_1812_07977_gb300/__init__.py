"""GB300-native finite-volume Euler step (the RiemannProblem fluid kernels of
Budiardja & Cardall, Sec. 3) behind a C ABI; see include/fv.h.

``Mesh`` (in ``fv``) is the binding; ``problems`` holds the seeded initial
conditions; ``build`` compiles the CUDA library in-tree.
"""
from . import problems  # noqa: F401

__all__ = ["problems", "Mesh", "FvError", "load_library", "build"]


def __getattr__(name):
    if name in ("Mesh", "FvError", "load_library"):
        from . import fv
        return getattr(fv, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
