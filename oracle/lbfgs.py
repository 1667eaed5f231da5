"""Oracle: quasi-Newton powered min-marginal averaging (Alg. 1 with Alg. 4, 5, 6), FP64.

Test infrastructure only (see ``oracle/__init__.py``). One call of ``QuasiNewton.step``
is one execution of Alg. 1 on the dual variables of a ``DualOracle``:

1. the deferred means are moved into lambda (lambda <- lambda + pend), so that the dual
   variables are the effective costs and pend = 0;
2. subgradient g: per BDD the minimising assignment of s^T lambda^j (Alg. 1, first line),
   per slot 1 iff the slot's min-marginal difference is negative (App. A.5 sign meaning);
3. direction d^ = H g by the L-BFGS two-loop recursion (Alg. 5), then the dual-feasible
   projection d^j_i = d^^j_i - mean over i's slots (Alg. 1, third line);
4. step size by the search of Alg. 6; the step is taken only if it raised the bound;
5. ``mma_iters`` deferred-MMA iterations (the first-order method, Alg. 1 "MMA");
6. the (s, y) pair of this call enters the L-BFGS memory if it passes the curvature test
   (Alg. 4).

Readings (the printed algorithms are partly garbled):
* L-BFGS is the textbook method applied to -E (minimisation), with the gradient of -E
  equal to -g: s_k = lambda_{k+1} - lambda_k and y_k = g(lambda_k) - g(lambda_{k+1}), so
  the curvature test s^T y >= eps (Alg. 4) is the usual one; the paper writes y with the
  opposite sign, under which the test could essentially never pass for a concave E.
* Alg. 5's second loop uses beta = rho_j y_j^T d (the printed "r" is the running d).
* Alg. 6 starts from E_init = E(lambda) (the printed E(lambda + gamma d) would make the
  first comparison trivially true); each of its K rounds evaluates E at the new step.
* Delta_min = 1e-6 (E(lambda^1) - E(lambda^0)) once the first call has finished; during
  the first call it is 0.
* Constants from the paper: eps = 1e-8, step growth 1.1, shrink 0.8, K = 5. Not stated
  in the paper and chosen here: memory m = 5, first step size 1e-3, 20 MMA iterations per
  call; lambda and b are reset consistently after a step (one backward min-sum pass).
"""
from __future__ import annotations

import numpy as np

from .solver import DualOracle


class QuasiNewton:
    def __init__(self, oracle: DualOracle, memory: int = 5, mma_iters: int = 20, eps: float = 1e-8,
                 grow: float = 1.1, shrink: float = 0.8, K: int = 5, gamma0: float = 1e-3):
        self.o = oracle
        self.m = int(memory)
        self.mma_iters = int(mma_iters)
        self.eps = float(eps)
        self.grow, self.shrink, self.K = float(grow), float(shrink), int(K)
        self.gamma = float(gamma0)
        self.S: list[np.ndarray] = []  # oldest first
        self.Y: list[np.ndarray] = []
        self.dmin = 0.0
        self.calls = 0
        self.E_start = None
        self.last = {}

    # ---- pieces ------------------------------------------------------------------------
    def bound(self, lam: np.ndarray) -> float:
        """E(lambda) + constant for per-slot dual variables with no deferred mean."""
        return float(self.o.bdd_minima(lam).sum()) + self.o.dec.const

    def subgradient(self, lam: np.ndarray) -> np.ndarray:
        return (self.o.min_marginals(lam) < 0).astype(np.float64)

    def direction(self, g: np.ndarray) -> np.ndarray:
        """H g by the two-loop recursion over the stored pairs (Alg. 5)."""
        q = g.copy()
        alphas = []
        for s, y in zip(reversed(self.S), reversed(self.Y)):  # newest first
            a = (s @ q) / (s @ y)
            q -= a * y
            alphas.append(a)
        if self.S:
            s, y = self.S[-1], self.Y[-1]
            q *= (s @ y) / (y @ y)
        for (s, y), a in zip(zip(self.S, self.Y), reversed(alphas)):  # oldest first
            b = (y @ q) / (s @ y)
            q += s * (a - b)
        return q

    def project(self, d: np.ndarray) -> np.ndarray:
        """Subtract each variable's mean over its slots: sum_j d^j_i = 0 (Eq. D feasibility)."""
        lv = self.o.lvar
        deg = self.o.dec.deg
        mean = np.bincount(lv, weights=d, minlength=len(deg)) / np.maximum(deg, 1)
        return d - mean[lv]

    def find_step(self, lam: np.ndarray, d: np.ndarray, E0: float) -> tuple[float, float]:
        """Alg. 6: returns (gamma_m, E(lambda + gamma_m d))."""
        gamma = self.gamma
        gm, Em = gamma, self.bound(lam + gamma * d)
        e = Em
        for _ in range(self.K):
            gamma = gamma * (self.shrink if e <= E0 else self.grow)
            e = self.bound(lam + gamma * d)
            if e >= Em:
                gm, Em = gamma, e
            if e - E0 >= self.dmin:
                break
        return gm, Em

    # ---- one call of Alg. 1 -----------------------------------------------------------------
    def step(self) -> None:
        o = self.o
        o.flush()
        lam = o.lam.copy()
        E0 = self.bound(lam)
        if self.E_start is None:
            self.E_start = E0
        g = self.subgradient(lam)
        d = self.project(self.direction(g))
        gm, Em = self.find_step(lam, d, E0)
        took = Em > E0
        if took:
            o.lam = lam + gm * d
        self.gamma = gm
        o.reset_b()
        o.iterate(self.mma_iters)
        lam_new = o.effective_costs()
        g_new = self.subgradient(lam_new)
        s = lam_new - lam
        y = g - g_new
        sy = float(s @ y)
        if sy >= self.eps:
            self.S.append(s)
            self.Y.append(y)
            if len(self.S) > self.m:
                self.S.pop(0)
                self.Y.pop(0)
        self.calls += 1
        if self.calls == 1:
            self.dmin = 1e-6 * (o.lower_bound() - self.E_start)
        self.last = {"E0": E0, "gamma": gm, "E_step": Em, "took": took, "sy": sy, "pairs": len(self.S)}
