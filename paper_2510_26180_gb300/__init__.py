"""GB300-native KLE-PCGC: Python binding of the sm_103a C-ABI library libklecgc.

Every step of the solve runs in the library's CUDA kernels; this package only
marshals arguments.  Importing it does not build anything; ``load()`` (called
by the binding on first use) fails loudly when the compiled library is
missing.
"""
from .klecgc import (FP64, MIXED, MIXED_DEFECT, GUESS_GPC, GUESS_ZERO, GUESS_USER,
                     GUESS_COARSE, GUESS_MLP, OK, E_INVALID_ARG, E_OUT_OF_MEMORY, E_NOT_CONVERGED,
                     E_NONFINITE, E_CUDA, E_UNSUPPORTED, KlecgcError, Problem, Solver, load,
                     exported_symbols, solve_batch, kl_basis, gpc_indices)

__all__ = ["FP64", "MIXED", "MIXED_DEFECT", "GUESS_GPC", "GUESS_ZERO", "GUESS_USER",
           "GUESS_COARSE", "GUESS_MLP", "OK", "E_INVALID_ARG", "E_OUT_OF_MEMORY", "E_NOT_CONVERGED",
           "E_NONFINITE", "E_CUDA", "E_UNSUPPORTED", "KlecgcError", "Problem", "Solver", "load",
           "exported_symbols", "solve_batch", "kl_basis", "gpc_indices"]
