"""FP64 CPU oracle for the rank-1-lattice sparse FFT (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The product path (``paper_2006_13053_gb300``) never does.
"""
from .sfft_oracle import *  # noqa: F401,F403
