"""CPU oracle for the compression-enabled processing model (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The product path (the CUDA library and its binding) never
does.  Every function here follows the paper's definitions; see ``oracle.c``.

Parity unpinned: none -- every oracle function is pinned by ``tests/test_oracle_pins.py``.
"""
from .oracle import *  # noqa: F401,F403
