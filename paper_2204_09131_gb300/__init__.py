"""GB300-native window-MI engine for iSYCOS (arXiv 2204.09131).

The compute path is the CUDA library ``libisycos.so`` (sources in ``csrc/``, C ABI in
``include/isycos.h``); :mod:`.api` is a thin ctypes binding with the same names.
:mod:`.synth` draws the seeded synthetic series used by tests and the benchmark.
"""
import importlib

__all__ = ["api", "synth"]


def __getattr__(name):
    if name in ("api", "synth", "build"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
