"""CPU oracle for the empty-space-skipping hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  The library product never does.
"""
from .oracle import *  # noqa: F401,F403
