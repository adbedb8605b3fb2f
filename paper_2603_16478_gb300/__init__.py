"""GB300-native analytical adjoint of one implicit step of a Neo-Hookean tet mesh with
smoothed Signorini-Coulomb contact ("Fast and Reliable Gradients for Deformables Across
Frictional Contact Regimes").

The compute path is the C-ABI library ``libncpadj.so`` (hand-written CUDA for sm_103a, declared
in ``include/ncpadj.h``); this package only marshals arguments to it.  There is no CPU
fallback: every call fails loudly if the library is not built.
"""
from .binding import (BatchCall, Bindings, Contacts, Context, Scene, NcpadjError, adjoint_batch, adjoint_step, elastic_solve,
                      forward_step, library_path, load_library, status_name)

__all__ = ["BatchCall", "Bindings", "Contacts", "Context", "Scene", "NcpadjError", "adjoint_batch", "adjoint_step", "elastic_solve",
           "forward_step", "library_path", "load_library", "status_name"]
