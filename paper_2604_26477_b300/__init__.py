"""B300 library for multi-objective MaxCut sampling by noise-injected simulated
bifurcation (arXiv 2604.26477): C ABI ``libmoqaia.so`` (``include/moqaia.h``), its
binding ``moqaia``, a round driver ``pipeline`` and the seeded input generators
``workloads``.

Importing the package loads nothing; ``moqaia`` and ``pipeline`` load the CUDA
library on first import and raise if it is missing.
"""
import importlib

__all__ = ["moqaia", "pipeline", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
