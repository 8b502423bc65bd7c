"""FP64 CPU oracle of the Phurbas particle RHS.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline leg / reference arm are the only users.  See oracle/oracle.py.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import __all__  # noqa: F401
