"""GB300-native (sm_103a) FFT bin-averaged 3D bispectrum estimator (arXiv:2107.14564, Sec. 2).

The compute path is the CUDA library libbispec.so (C ABI in include/bispec.h); this package is
its thin Python binding. Importing the package does not load the library; the first call does,
and raises if the library has not been built (`python -m paper_2107_14564_gb300.build`).
"""
__all__ = ["Plan", "BispecError", "binding", "build"]


def __getattr__(name):
    if name in ("Plan", "BispecError"):
        from . import binding
        return getattr(binding, name)
    if name in ("binding", "build", "autograd"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
