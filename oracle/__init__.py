"""FP64 CPU oracle for the one-loop SIAM fRG flow (test infrastructure only).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
import this package.  It shares no code with the CUDA path.
"""
from .oracle import (Model, rhs, rhs_rows, rhs_entries, flow, propagators,
                     observables, dp5_tableau, dp5_integrate, set_threads,
                     max_threads, MASK_TAILS, TAIL_FACTOR)

__all__ = ["Model", "rhs", "rhs_rows", "rhs_entries", "flow", "propagators",
           "observables", "dp5_tableau", "dp5_integrate", "set_threads",
           "max_threads", "MASK_TAILS", "TAIL_FACTOR"]
