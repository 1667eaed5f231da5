"""Oracle: exact ILP optimum of tiny instances by exhaustive search.

Test infrastructure only (see ``oracle/__init__.py``). Pins the dual bound
(LB <= OPT, weak duality of Eq. D) and the primal heuristic on
tetrahedron-sized problems.

Depth-first search: propagate all rows of (P) to generalised arc consistency,
prune with the cost of the variables already at 1 (costs are >= 0), branch on
the first X-triangle projection row that has no variable at 1 by setting each
of its free variables to 1 in turn.
"""
from __future__ import annotations

import numpy as np

from .problem import Infeasible, Problem, gac


def solve_exact(prob: Problem, node_limit: int = 200000):
    """Returns (opt_cost, x, n_optimal_solutions_found, nodes)."""
    assert np.all(prob.cost >= 0)
    best = [np.inf, None, 0]
    nodes = [0]
    xrows = range(prob.n_closed, prob.n_closed + prob.n_projx)

    def dfs(fixed):
        nodes[0] += 1
        if nodes[0] > node_limit:
            raise RuntimeError("node limit")
        try:
            fixed = gac(prob, fixed)
        except Infeasible:
            return
        part = float(prob.cost[fixed == 1].sum())
        if part > best[0] + 1e-12:
            return
        for r in xrows:
            v, _, _ = prob.row(r)
            if not np.any(fixed[v] == 1):
                for var in v[fixed[v] < 0]:
                    f2 = fixed.copy()
                    f2[var] = 1
                    dfs(f2)
                return
        # every X triangle covered once; GAC fixed everything else
        if np.any(fixed < 0):
            # still free variables: finish them by branching on any
            var = int(np.nonzero(fixed < 0)[0][0])
            for v in (0, 1):
                f2 = fixed.copy()
                f2[var] = v
                dfs(f2)
            return
        x = fixed.astype(np.int64)
        assert not np.any(prob.residual(x))
        c = float(prob.cost @ x)
        if c < best[0] - 1e-12:
            best[0], best[1], best[2] = c, x.copy(), 1
        elif abs(c - best[0]) <= 1e-12:
            best[2] += 1

    dfs(-np.ones(prob.nvars, np.int8))
    return best[0], best[1], best[2], nodes[0]


def lp_relaxation(prob: Problem):
    """Optimum of the LP relaxation of (P) (scipy HiGHS), or None if scipy is unavailable.

    Each row is a single +-1 equality, totally unimodular on its own, so the maximum
    of the dual (D) equals this LP optimum (for the unsplit decomposition)."""
    try:
        from scipy.optimize import linprog
        from scipy.sparse import csr_matrix
    except Exception:  # pragma: no cover
        return None
    A = csr_matrix((prob.row_coef.astype(float), prob.row_var, prob.row_ptr), shape=(prob.nrows, prob.nvars))
    res = linprog(prob.cost, A_eq=A, b_eq=prob.rhs.astype(float), bounds=(0, 1), method="highs")
    if res.status != 0:
        return None
    return float(res.fun)
