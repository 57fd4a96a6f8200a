"""GB300-native hot path of Pyramidal Gradient Matching (arXiv 1704.03217).

The method runs in libpgm.so (hand-written CUDA for sm_103a, C ABI in
include/pgm.h); this package only marshals arguments.  ``synth`` makes seeded
synthetic image pairs.  Importing the package does not load the library;
``api`` does, and raises if it is not built.
"""
import importlib

__all__ = ["api", "synth", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
