"""CPU oracle for the 2-forest / TTF Kemeny-constant method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library.  It shares
no code with the CUDA path.

Parity pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``
(closed forms, exhaustive spanning-tree enumeration, chi-square uniformity,
identities from the paper).  Nothing here is "parity unpinned".
"""
from .core import *  # noqa: F401,F403
from .exact import *  # noqa: F401,F403
from .blocktri import *  # noqa: F401,F403
from .hutchinson import *  # noqa: F401,F403
from .estimate import *  # noqa: F401,F403
