"""GB300-native (sm_103a) SHO projector library: projection, expansion and forces of real-space grid
wave functions on analytical 3D Hermite-Gauss projectors (Baumeister & Tsukamoto, PASC'19).

The compute path is libsho.so (CUDA kernels behind the C ABI of include/sho.h); this package binds it
for PyTorch tensors.  Importing the package does not load the library; the first call does, and fails
loudly if it has not been built.
"""
from ._native import ShoError  # noqa: F401

__all__ = ["ShoError", "api", "build"]


def __getattr__(name):
    if name in ("api", "build", "autograd", "serve"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
