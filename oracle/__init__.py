"""Plain CPU oracle for butterfly counting: test infrastructure only.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The product path (paper_1801_00338_gb300) never does.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, lib  # noqa: F401
