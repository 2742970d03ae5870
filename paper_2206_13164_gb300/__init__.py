"""GB300 (sm_103a) nonlinear multigrid solver for the regularized Hermite moment
discretization of rarefied cavity flow (Hu & Li, arXiv 2206.13164).

The compute path is the CUDA library ``libnrmg.so`` behind the C ABI ``include/nrmg.h``;
``paper_2206_13164_gb300.nrmg`` is its Python binding.
"""
from .nrmg import Solver, from_problem, lib, library_path, NrmgError  # noqa: F401
