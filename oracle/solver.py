"""Oracle: the dual iteration, lower bounds and min-marginals on explicit BDDs (FP64).

Test infrastructure only (see ``oracle/__init__.py``). The numeric loops live in
``oracle/mma.c`` (plain C, compiled with gcc on first use or by ``build()``).

Passages followed: Eq. D (dual and its feasibility constraint), Sec. 3.2
(shortest paths through BDDs), App. A.5 (min-marginal differences), Alg. 1
"MMA" line (first-order min-marginal averaging, deferred and parallel across
subproblems).

Readings (the paper leaves them to the cited first-order method):
* lambda^j_i starts at c_i / |J_i|, the deferred mass ``pend`` at 0, omega = 0.5;
  b is initialised by one backward min-sum pass without updates;
* one iteration = forward half-pass then backward half-pass, each followed by
  pend_i = (sum of the mass removed from i's slots) / |J_i|;
* the reported lower bound is E(lambda~) with lambda~^j_i = lambda^j_i + pend_i,
  a dual-feasible point of (D) (``lower_bound``);
* ``pool_bound`` = sum_j min_s s^T lambda^j + sum_i min(0, |J_i| pend_i) is the
  bound of the same decomposition with one extra unary subproblem per variable
  holding the deferred mass; every step of a half-pass moves mass between a
  subproblem and that pool without lowering it, so it never decreases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .bdd import Decomposition

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle_mma.so")
_lock = threading.Lock()
_lib = None


def build_c() -> str:
    """Compile ``mma.c`` with gcc into ``oracle/_build``."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "mma.c")
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build_c())
            _lib.or_half_pass.restype = ctypes.c_int64
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class DualOracle:
    """Sequential FP64 replay of the deferred-MMA dual iteration."""

    def __init__(self, dec: Decomposition, omega: float = 0.5):
        self.dec = dec
        self.omega = float(omega)
        self.lvar = dec.layer_var
        d = dec.deg[self.lvar].astype(np.float64)
        self.lam = dec.cost[self.lvar] / d
        self.pend = np.zeros(dec.nvars_total)
        self.f = np.zeros(dec.n_nodes)
        self.b = np.zeros(dec.n_nodes)
        self.state = None  # int8 per variable during rounding
        self.iterations = 0
        self.reset_b()

    # ---- raw passes -------------------------------------------------------------
    def _args(self):
        d = self.dec
        return (ctypes.c_int64(d.nb), _p(d.bdd_layer_ptr), _p(d.layer_var), _p(d.layer_node_ptr),
                _p(d.node_lo), _p(d.node_hi))

    def forward_minsum(self, cost: np.ndarray, state=None):
        f = np.zeros(self.dec.n_nodes)
        out = np.zeros(self.dec.nb)
        lib().or_forward(*self._args(), _p(np.ascontiguousarray(cost, np.float64)), _p(state), _p(f), _p(out))
        return f, out

    def backward_minsum(self, cost: np.ndarray, state=None):
        b = np.zeros(self.dec.n_nodes)
        out = np.zeros(self.dec.nb)
        lib().or_backward(*self._args(), _p(np.ascontiguousarray(cost, np.float64)), _p(state), _p(b), _p(out))
        return b, out

    def reset_b(self):
        self.b, _ = self.backward_minsum(self.lam, self.state)

    def half_pass(self, direction: int) -> None:
        acc = np.zeros(self.dec.nvars_total)
        bad = lib().or_half_pass(ctypes.c_int(direction), *self._args(), _p(self.lam), _p(self.pend), _p(acc),
                                 _p(self.state), ctypes.c_double(self.omega), _p(self.f), _p(self.b))
        if bad:
            raise FloatingPointError(f"{bad} layers with an infinite min-marginal")
        deg = self.dec.deg
        self.pend = np.where(deg > 0, acc / np.maximum(deg, 1), 0.0)

    def iterate(self, n: int = 1) -> None:
        for _ in range(n):
            self.half_pass(+1)
            self.half_pass(-1)
            self.iterations += 1

    # ---- bounds and marginals -----------------------------------------------------
    def effective_costs(self) -> np.ndarray:
        """lambda~ per layer: lambda plus the deferred mean."""
        return self.lam + self.pend[self.lvar]

    def bdd_minima(self, cost=None) -> np.ndarray:
        _, out = self.forward_minsum(self.effective_costs() if cost is None else cost, self.state)
        return out

    def lower_bound(self) -> float:
        """E(lambda~) + constant of fixed variables (Eq. D objective)."""
        return float(self.bdd_minima().sum()) + self.dec.const

    def pool_bound(self) -> float:
        m = self.bdd_minima(self.lam).sum()
        unary = np.minimum(0.0, self.dec.deg * self.pend).sum()
        return float(m + unary) + self.dec.const

    def min_marginals(self, cost=None, state=None) -> np.ndarray:
        """M per layer (slot) on lambda~ (or the given costs): min over s_i = 1 minus min over s_i = 0."""
        cost = self.effective_costs() if cost is None else cost
        f, _ = self.forward_minsum(cost, state)
        b, _ = self.backward_minsum(cost, state)
        m0 = np.zeros(self.dec.n_layers)
        m1 = np.zeros(self.dec.n_layers)
        d = self.dec
        lib().or_min_marginals(ctypes.c_int64(d.n_layers), _p(d.layer_node_ptr), _p(d.node_lo), _p(d.node_hi),
                               _p(np.ascontiguousarray(cost, np.float64)), _p(f), _p(b), _p(m0), _p(m1))
        return m1 - m0

    def feasibility_residual(self) -> np.ndarray:
        """sum_j lambda^j_i + |J_i| pend_i - c_i per variable (zero up to rounding)."""
        s = np.bincount(self.lvar, weights=self.lam, minlength=self.dec.nvars_total)
        return s + self.dec.deg * self.pend - np.where(self.dec.deg > 0, self.dec.cost, 0.0)

    def flush(self) -> None:
        """Move the deferred mean into every slot: lambda <- lambda~, pend <- 0."""
        self.lam = self.effective_costs()
        self.pend = np.zeros_like(self.pend)

    # ---- propagation ----------------------------------------------------------------
    def supports(self, state: np.ndarray):
        d = self.dec
        rf = np.zeros(d.n_nodes, np.int8)
        rb = np.zeros(d.n_nodes, np.int8)
        s0 = np.zeros(d.n_layers, np.int8)
        s1 = np.zeros(d.n_layers, np.int8)
        lib().or_supports(*self._args(), _p(state), _p(rf), _p(rb), _p(s0), _p(s1))
        return s0.astype(bool), s1.astype(bool)


def run_dual(dec: Decomposition, iters: int, omega: float = 0.5, lb_every: int = 0):
    """Convenience: iterate and record (iteration, E(lambda~), pool bound) every ``lb_every``."""
    o = DualOracle(dec, omega)
    trace = [(0, o.lower_bound(), o.pool_bound())]
    for t in range(1, iters + 1):
        o.iterate(1)
        if lb_every and (t % lb_every == 0 or t == iters):
            trace.append((t, o.lower_bound(), o.pool_bound()))
    return o, trace
