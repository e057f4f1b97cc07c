"""FP64 CPU oracle for the layer-split time stepper.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
use it.  It shares no code, tables or constants with the CUDA path.

See ``oracle/lsplit.py`` for the implementation and the paper passages each
function follows.
"""
from .lsplit import *  # noqa: F401,F403
