"""GB300-native polynomial-filtered subspace extraction (libpf).

The compute path is the CUDA library ``_lib/libpf.so`` (sources in ``csrc/``,
C ABI in ``include/pf.h``); :mod:`._binding` exposes its entry points under
the same names and :mod:`.solver` wraps them for PyTorch tensors (device
memory and streams only).  The binding loads on first use, so
``paper_1904_10585_gb300.build`` can run before the library exists; using
any entry point without the library raises ImportError (no CPU fallback).
"""
import importlib


_SUBMODULES = ("build", "solver", "_binding")


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    if name in _SUBMODULES:
        return importlib.import_module("." + name, __name__)
    binding = importlib.import_module("._binding", __name__)
    try:
        return getattr(binding, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
