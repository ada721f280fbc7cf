"""GB300 (sm_103a) implementation of the Birkhoff trajectory-optimisation hot path of
arXiv 2509.01855: matrix-free Birkhoff products, KKT operator, Birkhoff preconditioner,
right-preconditioned GMRES and the Newton driver, behind the C ABI of include/birkhoff.h.

The Python layer (``api``) only marshals arguments to ``libbirkhoff.so``.
"""
from .api import (Plan, Problem, birkhoff_apply, birkhoff_apply_T, kkt_apply, precond_apply,
                  krylov_solve, newton_solve)

__all__ = ["Plan", "Problem", "birkhoff_apply", "birkhoff_apply_T", "kkt_apply",
           "precond_apply", "krylov_solve", "newton_solve"]
