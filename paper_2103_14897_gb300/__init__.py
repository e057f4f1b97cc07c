"""GB300-native layer-split time stepper for the lifted plane-wave
Schroedinger equation of incommensurate bilayers (arXiv 2103.14897).

The computation runs in ``_lib/liblsplit.so`` (hand-written sm_103a CUDA
kernels behind the C ABI of ``include/lsplit.h``); this package holds the
ctypes binding, the build script and a ``torch.autograd.Function`` for
gradients of a final overlap with respect to the layer potentials.
"""
from ._binding import (Context, Batch, LsplitError, SCHEMES, EXPORTS, LIB_PATH, load_library,  # noqa: F401
                       LS_OK, LS_ERR_INVALID, LS_ERR_NOMEM, LS_ERR_CUDA, LS_ERR_TIMEOUT, LS_ERR_STATE)

__all__ = ["Context", "Batch", "LsplitError", "SCHEMES", "EXPORTS", "LIB_PATH", "load_library"]
