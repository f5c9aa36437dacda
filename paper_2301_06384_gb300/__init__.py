"""Block Krylov kernel columns phi(L) E_W on GB300 (arXiv 2301.06384).

The compute path is the C-ABI library ``libkb.so`` (``include/kb.h``), built from the CUDA
sources in ``csrc/``; ``kb`` is its ctypes binding.
"""
from . import kb  # noqa: F401
from .kb import (Graph, KbError, kb_graph_create, kb_krylov_apply, kb_krylov_apply_host,  # noqa: F401
                 kernel_columns, make_params)
