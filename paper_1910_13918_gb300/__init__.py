"""GB300-native semi-Lagrangian lattice Boltzmann step (arXiv:1910.13918).

``paper_1910_13918_gb300.sllbm``     Python binding of the C-ABI library (``include/sllbm.h``)
``paper_1910_13918_gb300.autograd``  checkpointed adjoint behind ``torch.autograd.Function``
``paper_1910_13918_gb300.workloads`` seeded synthetic workloads (input generators only)
``paper_1910_13918_gb300.build``     compiles the CUDA library for sm_103a

Importing the package loads nothing; the CUDA library is loaded on first use and a missing
library is an error, never a fallback.
"""
