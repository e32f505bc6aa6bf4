"""FP64 CPU oracle for the Hermitian-definite generalized eigenproblem.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``. The library's product path never imports it.
"""
from .oracle import *  # noqa: F401,F403
from . import pieces  # noqa: F401
