"""GB300-native row-wise assembly of isogeometric mass and stiffness matrices
with weighted Gaussian quadrature rules (one rule per row, the row's B-spline
as the measure), evaluated by sum factorisation into each row's band.

The compute path is the C-ABI library ``libwq.so`` (``include/wq.h``); the
Python names mirror its entry points and only marshal arguments.  Importing
this package does not load the library; the first call does, and fails
loudly if it has not been built.
"""
import importlib

_SUBMODULES = ("inputs", "binding", "build")


def __getattr__(name):
    if name in _SUBMODULES:
        return importlib.import_module(f"{__name__}.{name}")
    if name.startswith("__"):
        raise AttributeError(name)
    return getattr(importlib.import_module(f"{__name__}.binding"), name)
