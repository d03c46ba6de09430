"""FP64 CPU oracle for the pseudo-Verlet SPH density loop.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never imports
it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
