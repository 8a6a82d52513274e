"""CPU oracle for the KScaNN query path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs may
import this package.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
