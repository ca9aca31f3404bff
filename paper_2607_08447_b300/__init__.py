"""B300-native k.p hole eigensolver (the block eigensolve inside the
Schroedinger-Poisson loop of "Simulation of exchange coupling effects in
double quantum dot FinFET-like structures").

The compute path is the C-ABI library ``libkhp.so`` (include/khp.h) built
from ``csrc/`` for sm_103a; this package only marshals arguments.
"""
from ._lib import KHPError, load  # noqa: F401
from .solver import KPEigs, KPGrid, SolveResult, solve_batched  # noqa: F401
from .poisson import Poisson, SPResult, sp_solve  # noqa: F401
from .ci import CIResult, ci_detuning_sweep, ci_exchange  # noqa: F401
from .gtensor import GTensorResult, g_tensors  # noqa: F401
from . import exchange  # noqa: F401

__all__ = ["KPGrid", "KPEigs", "SolveResult", "solve_batched", "Poisson", "SPResult", "sp_solve",
           "CIResult", "ci_exchange", "ci_detuning_sweep", "GTensorResult", "g_tensors", "exchange",
           "KHPError", "load"]
