"""GB300-native symbolic-phase stabilizer sampler (arXiv 2311.03906).

The work runs in the CUDA library ``_build/libsymphase.so`` (C ABI in
include/symphase.h); this package is its Python binding."""
from .binding import (Program, SymPhaseError, batch_plans, build, debug_fail_alloc, debug_live_allocs, expect, load,
                      load_program, sample_batch, unpack_bits,
                      PATH_AUTO, PATH_DENSE, PATH_SPARSE, PATH_FUSED, PATH_TENSOR, EXPORTS, OPCODES)

__all__ = ["Program", "SymPhaseError", "batch_plans", "build", "debug_fail_alloc", "debug_live_allocs", "expect", "load", "load_program", "sample_batch", "unpack_bits",
           "PATH_AUTO", "PATH_DENSE", "PATH_SPARSE", "PATH_FUSED", "PATH_TENSOR", "EXPORTS",
           "OPCODES"]
