"""Plain FP64 CPU oracle for ECMG_jcg (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The CUDA library and its Python binding never do.
"""
from .oracle import *  # noqa: F401,F403
