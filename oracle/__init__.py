"""CPU oracle for the minimum distance of a binary linear code.

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the GPU library.
"""
from .oracle import *  # noqa: F401,F403
