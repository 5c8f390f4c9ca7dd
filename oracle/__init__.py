"""Plain FP64 CPU oracle for the multi-stage preconditioned FGMRES path.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import it. It shares no code
with the CUDA library and never serves as a fallback for it.
"""
from .oracle import (OracleAMG, OracleError, OracleSolver, colour, condense, interp_only,
                     options, pmis_rounds, recover, splitmix)

__all__ = ["OracleAMG", "OracleError", "OracleSolver", "colour", "condense", "interp_only",
           "options", "pmis_rounds", "recover", "splitmix"]
