"""Oracle: min-marginal-driven primal rounding with propagation.

Test infrastructure only (see ``oracle/__init__.py``).

Passages followed: primal recovery by the cited heuristic driven by this
paper's dual (Sec. 3 pipeline figure, Sec. 4 "Methods"); agreement semantics of
min-marginal signs, M^j_i > 0 means subproblem j prefers x_i = 0, all
subproblems with the same sign "agree" (App. A.5).

Reading (the paper defers the heuristic to its citation). Round r = 0 .. R-1:
  1. flush the deferred mean into lambda; compute M on the BDDs restricted to the
     current fixings;
  2. every free variable whose M^j_i are all > tau is fixed to 0, all < -tau to 1;
  3. propagate: in every BDD keep only values that lie on a root -> TOP path
     consistent with the fixings; fix variables left with one value, repeat to a
     fixpoint; a variable with no value left is a conflict, and then the whole
     round's fixings are undone;
  4. stop when every variable is fixed;
  5. perturb every free variable's slots by delta_r * sgn(sum_j M^j_i)
     (sgn(0) = +1, i.e. towards 0), delta_r = delta_0 * growth^r;
  6. recompute b under the fixings and run ``inner`` dual iterations on the
     restricted BDDs (fixed variables take no update).
Constants: tau = 1e-6, delta_0 = 1e-3, growth = 2, inner = 20, R = 100.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .problem import Problem
from .solver import DualOracle

FREE, FIX0, FIX1 = 0, 1, 2


@dataclass
class PrimalResult:
    x: np.ndarray  # (nvars,) uint8 of the original variables
    ok: bool
    cost: float
    rounds: int


def propagate(o: DualOracle, state: np.ndarray) -> bool:
    """Fix forced variables to a fixpoint. Returns False on a conflict."""
    lvar = o.lvar
    n = o.dec.nvars_total
    while True:
        s0, s1 = o.supports(state)
        # a value is possible for i iff every slot of i supports it
        bad0 = np.bincount(lvar, weights=~s0, minlength=n) > 0
        bad1 = np.bincount(lvar, weights=~s1, minlength=n) > 0
        inb = o.dec.deg > 0
        can0 = inb & ~bad0
        can1 = inb & ~bad1
        if np.any(inb & (state == FIX0) & ~can0) or np.any(inb & (state == FIX1) & ~can1):
            return False
        free = inb & (state == FREE)
        if np.any(free & ~can0 & ~can1):
            return False
        f1 = free & ~can0
        f0 = free & ~can1
        if not (f1.any() or f0.any()):
            return True
        state[f1] = FIX1
        state[f0] = FIX0


def round_primal(o: DualOracle, prob: Problem, fixed_presolve: np.ndarray, tau: float = 1e-6,
                 delta0: float = 1e-3, growth: float = 2.0, inner: int = 20, rounds: int = 100) -> PrimalResult:
    dec = o.dec
    n = dec.nvars_total
    inb = dec.deg > 0
    state = np.full(n, FREE, np.int8)
    o.state = state
    delta = delta0
    lvar = o.lvar
    r = 0
    for r in range(rounds):
        o.flush()
        M = o.min_marginals(o.lam, state)
        free_slot = state[lvar] == FREE
        pos = np.bincount(lvar, weights=free_slot & (M > tau), minlength=n)
        neg = np.bincount(lvar, weights=free_slot & (M < -tau), minlength=n)
        cnt = dec.deg
        free = inb & (state == FREE)
        trial = state.copy()
        trial[free & (pos == cnt)] = FIX0
        trial[free & (neg == cnt)] = FIX1
        if propagate(o, trial):
            state[:] = trial
        if not np.any(inb & (state == FREE)):
            break
        msum = np.bincount(lvar, weights=np.where(free_slot, M, 0.0), minlength=n)
        sgn = np.where(msum >= 0, 1.0, -1.0)
        upd = (state[lvar] == FREE)
        o.lam = o.lam + np.where(upd, delta * sgn[lvar], 0.0)
        delta *= growth
        o.reset_b()
        o.iterate(inner)
    else:
        r = rounds
    o.state = None
    x = np.where(fixed_presolve >= 0, fixed_presolve, 0).astype(np.uint8)
    orig = np.arange(prob.nvars)
    bvar = orig[inb[: prob.nvars]]
    x[bvar] = (state[bvar] == FIX1).astype(np.uint8)
    done = not np.any(inb & (state == FREE))
    ok = done and not np.any(prob.residual(x))
    cost = float(np.dot(prob.cost, x.astype(np.float64)))
    return PrimalResult(x, ok, cost, r + 1 if done else rounds)
