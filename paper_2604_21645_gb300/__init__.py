"""GB300-native product quantization (PQ) and IVF-ADC search.

The compute path lives in ``libpqgb.so`` (hand-written sm_103a CUDA behind a C
ABI, declared in ``include/pqgb.h``); :mod:`paper_2604_21645_gb300.pqgb` is the
ctypes binding with the same entry-point names.  Importing this package does
not load the library; the binding is imported on first attribute access.
"""
import importlib

__all__ = ["pqgb", "datagen", "softpq"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
