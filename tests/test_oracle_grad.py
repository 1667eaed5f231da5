"""Pins of the gradient oracle (``oracle/grad.py``): its bound equals the C oracle's after
the same iterations, and its autograd gradient equals central finite differences of the
C oracle (an independent implementation) along random directions; a planted mistake
in the replica is caught."""
import numpy as np
import pytest

from oracle import bdd as B
from oracle import grad as G
from oracle import problem as P
from oracle import solver as S
from synth import instances as I


def _dec(name, chunk):
    inst = getattr(I, name)()
    prob, d, allowed = P.make_problem(inst)
    fixed, const = P.presolve(prob)
    return prob, fixed, B.decompose(prob, fixed, const, chunk)


def _c_oracle_bound(dec, fixed, c, iters):
    d2 = B.Decomposition(**{**dec.__dict__, "cost": np.concatenate([c, np.zeros(dec.nvars_total - dec.nvars)]),
                            "const": float(c[fixed == 1].sum())})
    o = S.DualOracle(d2)
    o.iterate(iters)
    return o.lower_bound()


@pytest.mark.parametrize("name,chunk,iters", [("tet", 0, 30), ("tet", 3, 25), ("config1", 4, 6)])
def test_bound_matches_c_oracle_and_gradient_matches_differences(name, chunk, iters):
    prob, fixed, dec = _dec(name, chunk)
    lb, g = G.bound_and_grad(dec, prob.cost, fixed, iters)
    ref = _c_oracle_bound(dec, fixed, prob.cost, iters)
    assert abs(lb - ref) <= 1e-12 * max(1.0, abs(ref))
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(prob.nvars)
        eps = 1e-6
        fd = (_c_oracle_bound(dec, fixed, prob.cost + eps * v, iters) -
              _c_oracle_bound(dec, fixed, prob.cost - eps * v, iters)) / (2 * eps)
        assert abs(fd - float(g @ v)) <= 1e-6 * max(1.0, abs(fd))
    # fixed-to-1 variables enter through the constant, fixed-to-0 ones not at all
    assert np.all(g[fixed == 1] == 1.0) and np.all(g[fixed == 0] == 0.0)


def test_zero_iterations_gradient_is_mean_argmin_indicator():
    """With no iteration the bound is sum_j min_s s^T c / |J|: its gradient in c_i is the
    number of BDDs whose shortest path sets x_i = 1, divided by |J_i| (generic costs)."""
    prob, fixed, dec = _dec("tet", 0)
    lb, g = G.bound_and_grad(dec, prob.cost, fixed, 0)
    o = S.DualOracle(dec)
    lam = o.lam.copy()
    mm = o.min_marginals(lam)  # M < 0: every shortest path of that BDD takes the 1-arc
    ones = np.bincount(dec.layer_var, weights=(mm < 0).astype(float), minlength=dec.nvars_total)
    free = dec.deg[: dec.nvars] > 0
    np.testing.assert_allclose(g[free], (ones[: dec.nvars] / np.maximum(dec.deg[: dec.nvars], 1))[free], atol=1e-12)


def test_planted_mistake_is_caught():
    """A replica whose half-pass forgets the deferred mean drifts from the C oracle."""
    prob, fixed, dec = _dec("tet", 0)
    ud = G.UnrolledDual(dec)
    good = ud.half_pass

    def bad(lam, pend, other, forward):
        return good(lam, pend * 0.0, other, forward)

    ud.half_pass = bad
    import torch

    c = torch.tensor(np.concatenate([prob.cost, np.zeros(dec.nvars_total - dec.nvars)]))
    lb_bad = float(ud.lower_bound(c, 10)) + float(prob.cost[fixed == 1].sum())
    ref = _c_oracle_bound(dec, fixed, prob.cost, 10)
    assert abs(lb_bad - ref) > 1e-9
