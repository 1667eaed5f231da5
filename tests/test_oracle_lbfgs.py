"""Pins of the quasi-Newton oracle (``oracle/lbfgs.py``, Alg. 1 with Alg. 4-6).

* the two-loop recursion equals the product with the inverse-Hessian matrix built by the
  explicit BFGS update formula from the same pairs (textbook identity);
* the projection makes every variable's direction entries sum to 0 and is idempotent;
* the step search returns the best step it evaluated and follows the grow / shrink rule
  on a one-dimensional concave model;
* a call never lowers the bound, and only pairs passing the curvature test are stored.
"""
import numpy as np
import pytest

from oracle import bdd as B
from oracle import lbfgs as Q
from oracle import problem as P
from oracle import solver as S
from synth import instances as I


def _qn(name="config1", chunk=0, **kw):
    inst = getattr(I, name)()
    prob, d, allowed = P.make_problem(inst)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, chunk)
    return Q.QuasiNewton(S.DualOracle(dec), **kw)


def test_two_loop_equals_explicit_bfgs_inverse():
    rng = np.random.default_rng(0)
    n, m = 12, 4
    qn = Q.QuasiNewton.__new__(Q.QuasiNewton)
    qn.S, qn.Y = [], []
    A = rng.standard_normal((n, n))
    Hess = A @ A.T + n * np.eye(n)  # positive definite model curvature
    for _ in range(m):
        s = rng.standard_normal(n)
        qn.S.append(s)
        qn.Y.append(Hess @ s)  # s^T y > 0
    g = rng.standard_normal(n)
    s, y = qn.S[-1], qn.Y[-1]
    H = (s @ y) / (y @ y) * np.eye(n)
    for s, y in zip(qn.S, qn.Y):  # oldest first
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    np.testing.assert_allclose(qn.direction(g), H @ g, rtol=1e-10, atol=1e-12)
    qn.S, qn.Y = [], []
    np.testing.assert_array_equal(qn.direction(g), g)  # no pairs: identity


def test_projection_is_dual_feasible_and_idempotent():
    qn = _qn("tet")
    rng = np.random.default_rng(1)
    d = rng.standard_normal(qn.o.dec.n_layers)
    p = qn.project(d)
    sums = np.bincount(qn.o.lvar, weights=p, minlength=qn.o.dec.nvars_total)
    np.testing.assert_allclose(sums, 0.0, atol=1e-12)
    np.testing.assert_allclose(qn.project(p), p, atol=1e-12)


def test_step_search_on_concave_model():
    qn = Q.QuasiNewton.__new__(Q.QuasiNewton)
    qn.gamma, qn.grow, qn.shrink, qn.K, qn.dmin = 1.0, 1.1, 0.8, 5, 1e9
    best = 2.0  # E(lambda + gamma d) = 1 - (gamma - 2)^2, E(lambda) = -10
    evals = []

    def bound(x):
        gam = float(x[0])
        evals.append(gam)
        return 1.0 - (gam - best) ** 2

    qn.bound = bound
    gm, Em = qn.find_step(np.zeros(1), np.ones(1), -10.0)
    # improving steps grow by 1.1 each round: 1.1, 1.21, ... ; the best evaluated is returned
    assert evals[0] == 1.0
    np.testing.assert_allclose(evals[1:], [1.1 ** k for k in range(1, 6)], rtol=1e-12)
    assert gm == pytest.approx(max(evals, key=lambda g: 1.0 - (g - best) ** 2))
    assert Em == pytest.approx(1.0 - (gm - best) ** 2)
    # a step that does not improve shrinks
    evals.clear()
    qn.gamma = 6.0  # E = -15 < -10
    gm, Em = qn.find_step(np.zeros(1), np.ones(1), -10.0)
    assert evals[1] == pytest.approx(4.8)
    # sufficient improvement stops the search
    evals.clear()
    qn.gamma, qn.dmin = 1.0, 5.0
    qn.find_step(np.zeros(1), np.ones(1), -10.0)
    assert len(evals) == 2


@pytest.mark.parametrize("name,chunk", [("config1", 0), ("config1", 4)])
def test_calls_never_lower_the_bound(name, chunk):
    qn = _qn(name, chunk, mma_iters=3)
    lb = qn.o.lower_bound()
    for _ in range(5):
        qn.step()
        nxt = qn.o.lower_bound()
        assert nxt >= lb - 1e-12 * max(1.0, abs(lb))
        lb = nxt
        assert all(float(s @ y) >= qn.eps for s, y in zip(qn.S, qn.Y))
        assert len(qn.S) <= qn.m
    # dual feasibility is kept exactly through the quasi-Newton steps
    np.testing.assert_allclose(qn.o.feasibility_residual(), 0.0, atol=1e-12)
