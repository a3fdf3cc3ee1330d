"""GB300-native nonsmooth sphere DEM step for locally refined beds (arXiv 2501.05300).

The simulation runs in libdem.so (CUDA, sm_103a) behind the C ABI of
include/dem.h; `dem` is its Python binding, `beds` builds seeded synthetic
inputs and `rules` holds the paper's host-side set-up rules (Eqs. 1, 8-10).
"""
from . import beds, rules  # noqa: F401


def build(force: bool = False) -> str:
    """Compile libdem.so for sm_103a; returns its path."""
    from . import buildlib as _b
    return _b.build(force=force)


def __getattr__(name):
    if name == "Bed":
        import importlib
        return importlib.import_module(__name__ + ".dem").Bed
    raise AttributeError(name)
