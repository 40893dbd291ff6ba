"""FP64 CPU oracle for the ISM hot path.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The product path never routes through it.
"""
from . import ism_oracle  # noqa: F401
