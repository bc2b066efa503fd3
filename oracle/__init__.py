"""CPU float64 oracle for Exp-ParaDiag -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may import, call or execute anything under this package.  It shares no code
with the CUDA path (paper_2603_04350_gb300) and neither imports the other.
"""
from .expd_oracle import *  # noqa: F401,F403
from .expd_oracle import Spec, spec_of, bdf_coefficients, bdf_float  # noqa: F401
