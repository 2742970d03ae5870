"""GB300 (sm_103a) nonlinear multigrid solver for the regularized Hermite moment
discretization of rarefied cavity flow (Hu & Li, arXiv 2206.13164).

The compute path is the CUDA library ``libnrmg.so`` behind the C ABI ``include/nrmg.h``
(solver, batches) and ``include/nrmg_net.h`` (the learned start's network and field glue).
``paper_2206_13164_gb300.nrmg`` binds the solver (``Solver``, ``Batch``);
``paper_2206_13164_gb300.learned`` binds the network (``Net``) and sequences the learned
start (``LearnedSolve``) and its training.
"""
from .nrmg import Batch, NrmgError, Solver, from_problem, lib, library_path  # noqa: F401
