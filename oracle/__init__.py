"""FP64 CPU oracle for the HJ safe-set solve.

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py; never by the CUDA product path.
"""
from .binding import *  # noqa: F401,F403
from .binding import build, lib  # noqa: F401
