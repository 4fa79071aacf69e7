"""GB300-native lattice core-Hamiltonian solver (arXiv:1408.3839): assembly of the core
Hamiltonian and overlap of a lattice Gaussian basis from weighted 1D Gram contractions, block
DFT along the lattice indices, and k-point generalized Hermitian eigensolves -- all in the
CUDA library liblhf.so (C ABI in include/lhf.h).  ``paper_1408_3839_gb300.lhf`` is the thin
Python binding (argument marshalling only)."""

from .lhf import (FP64, MIXED, LHF_OK, LHF_ERR_ARG, LHF_ERR_CUDA, LHF_ERR_NOT_SPD,  # noqa: F401
                  LHF_ERR_STATE, LHF_ERR_UNSUPPORTED, Context, LhfError, library_path, load)
