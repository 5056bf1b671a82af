"""CPU oracle for ST-HOSVD (test infrastructure; never used by the product path).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  It shares no code with the CUDA
library under ``paper_1510_06689_gb300/``.
"""
from .st_hosvd import *  # noqa: F401,F403
from .st_hosvd import __all__  # noqa: F401
