"""GB300-native stress-velocity Newton (svN) solver for the implicit
viscous-plastic sea-ice momentum step (arXiv:2204.10822).

The compute path is the CUDA library ``libsvn.so`` (C ABI in
``include/svn.h``); this package only marshals arguments.  PyTorch provides
device memory and streams.
"""
from .solver import Batch, Q2Solver, Solver, SvnError, default_params  # noqa: F401
