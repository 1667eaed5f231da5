"""GB300-native (sm_103a) DiscoMatch dual / primal solver.

The hot path — pair costs, candidate mask, BDD min-sum passes, deferred
min-marginal averaging, lower bound, rounding — runs in hand-written CUDA
kernels behind the C ABI of ``include/disco.h``; ``_lib`` binds it with ctypes
and ``api`` wraps it for NumPy / PyTorch callers. There is no CPU fallback: a
missing library raises.
"""
from .api import Solver, candidates, pair_costs  # noqa: F401
