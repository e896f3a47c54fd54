"""GB300-native D2Q9 improved-MRT pseudopotential lattice Boltzmann (arXiv:1211.6932).

The computation lives in the CUDA library ``liblbm_gb300.so`` (C ABI in include/lbm.h);
this package only marshals arguments to it.  Import is lazy: the library is loaded on
first use of ``Lattice``/``Batch`` and loading fails loudly if it has not been built.
"""

__all__ = ["Lattice", "Batch", "Eos", "maxwell", "lib", "LbmError", "Mlp"]


def __getattr__(name):
    if name in ("Lattice", "Batch", "Eos", "maxwell", "LbmError", "Options", "Instance"):
        from . import lattice
        return getattr(lattice, name)
    if name == "Mlp":
        from . import mlp
        return mlp.Mlp
    if name == "lib":
        from . import _lib
        return _lib.lib
    raise AttributeError(name)
