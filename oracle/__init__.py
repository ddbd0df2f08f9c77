"""Plain CPU oracle of the symbolic-phase sampler (test infrastructure only)."""
from .oracle import (Program, OracleError, build, philox4x32_10, threshold, unpack_records,
                     circuit_arrays, CH_TYPES)

__all__ = ["Program", "OracleError", "build", "philox4x32_10", "threshold", "unpack_records",
           "circuit_arrays", "CH_TYPES"]
