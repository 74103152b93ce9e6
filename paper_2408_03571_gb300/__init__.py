"""GB300 (sm_103a) two-level Schwarz preconditioned GMRES for the 2-D Helmholtz equation.

Method: "Coarse Spaces Based on Higher-Order Interpolation for Schwarz
Preconditioners for Helmholtz Problems" (arXiv 2408.03571): second-order
finite differences for MP-1 (Dirichlet) and MP-2 (Sommerfeld), overlapping
Schwarz preconditioners AS1 / AS2 / SAS2 / SHS2 with P_1 or B_2 coarse spaces,
solved by GMRES.  The computation lives in ``libhzs.so`` (CUDA, C ABI in
``include/hzs.h``); :mod:`.hzs` is its ctypes binding and :mod:`.autograd`
the differentiable wrapper.  Submodules are imported lazily so that the input
generators (:mod:`.inputs`) load without torch or the CUDA library.
"""
import importlib

__all__ = ["hzs", "inputs", "autograd", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
