"""Pins of the oracle's min-sum, min-marginals, dual iteration and primal rounding (CPU).

Eq. D (dual, feasibility, weak duality), App. A.5 (min-marginal differences),
Alg. 1 "MMA" (non-decreasing first-order updates), Sec. 4 (optimality gaps)."""
import itertools

import numpy as np
import pytest

from oracle import bdd as B
from oracle import exact as E
from oracle import primal as PR
from oracle import problem as P
from oracle import solver as S
from synth import instances as I


def _single_row_dec(coef, rhs, chunk=0):
    n = len(coef)
    bdd, _ = B.compile_row(np.arange(n), np.asarray(coef), rhs)
    segs, aux, nxt = B.split_row(bdd, chunk, n)
    return B.flatten(segs, [0] * len(segs), n, nxt, np.zeros(nxt), np.ones(n, bool), 0.0), segs, aux


def _brute(segs, cost, nvar):
    """All joint assignments accepted by every segment, with their costs."""
    vars_ = sorted({v for s in segs for v in s.var})
    out = []
    for vals in itertools.product([0, 1], repeat=len(vars_)):
        a = dict(zip(vars_, vals))
        if all(s.evaluate(a) for s in segs):
            out.append(a)
    return out


@pytest.mark.parametrize("seed", range(5))
def test_min_marginals_match_brute_force(seed):
    """M^j_i = min_{s_i=1} s^T l - min_{s_i=0} s^T l per BDD (App. A.5) against enumeration."""
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(15):
        n = int(rng.integers(2, 11))
        coef = rng.choice([-1, 1], n)
        vals = {int(np.dot(coef, s)) for s in itertools.product([0, 1], repeat=n)}
        rhs = int(rng.choice(sorted(vals)))
        dec, segs, aux = _single_row_dec(coef, rhs)
        o = S.DualOracle.__new__(S.DualOracle)
        o.dec = dec
        o.lvar = dec.layer_var
        cost = rng.standard_normal(dec.n_layers)
        M = o.min_marginals(cost)
        _, mins = o.forward_minsum(cost)
        sols = [np.array(s) for s in itertools.product([0, 1], repeat=n) if np.dot(coef, s) == rhs]
        vals_ = [float(np.dot(cost, s)) for s in sols]
        assert mins[0] == pytest.approx(min(vals_), abs=1e-12)
        for i in range(n):
            m1 = min([v for v, s in zip(vals_, sols) if s[i] == 1], default=np.inf)
            m0 = min([v for v, s in zip(vals_, sols) if s[i] == 0], default=np.inf)
            assert M[i] == pytest.approx(m1 - m0, abs=1e-12)


def test_exactly_one_min_marginals_closed_form():
    """For sum_i x_i = 1: M_i = l_i - min_{k != i} l_k."""
    rng = np.random.Generator(np.random.PCG64(9))
    for n in (2, 3, 7, 40):
        dec, _, _ = _single_row_dec(np.ones(n, np.int64), 1)
        o = S.DualOracle.__new__(S.DualOracle)
        o.dec = dec
        o.lvar = dec.layer_var
        lam = rng.standard_normal(n)
        M = o.min_marginals(lam)
        ref = np.array([lam[i] - np.min(np.delete(lam, i)) for i in range(n)])
        np.testing.assert_allclose(M, ref, atol=1e-12)


@pytest.mark.parametrize("chunk", [2, 3])
def test_split_min_marginals_of_originals_match_joint_brute_force(chunk):
    """Min over the joint feasible set of split segments with the aux cost split evenly
    equals the unsplit row's minimum (equivalence, App. A.3)."""
    rng = np.random.Generator(np.random.PCG64(chunk))
    coef = np.array([1, 1, -1, 1, -1, 1, 1])
    dec, segs, aux = _single_row_dec(coef, 1, chunk)
    x_cost = rng.standard_normal(7)
    sols = _brute(segs, None, None)
    best = min(sum(x_cost[v] * a[v] for v in range(7)) for a in sols)
    ref = min(float(np.dot(x_cost, s)) for s in itertools.product([0, 1], repeat=7) if np.dot(coef, s) == 1)
    assert best == pytest.approx(ref, abs=1e-12)


def _lb0_brute(prob, dec):
    """E(lambda^0): sum over rows of the row minimum of c_i/|J_i|, by enumeration for
    closedness rows and by the closed form min_i lambda_i for the exactly-one rows."""
    lam_var = np.where(dec.deg[: prob.nvars] > 0, prob.cost / np.maximum(dec.deg[: prob.nvars], 1), 0)
    tot = 0.0
    for r in range(prob.nrows):
        v, a, rhs = prob.row(r)
        if r >= prob.n_closed:
            tot += float(lam_var[v].min())
            continue
        assert len(v) <= 16
        best = np.inf
        for s in itertools.product([0, 1], repeat=len(v)):
            if np.dot(a, s) == rhs:
                best = min(best, float(np.dot(lam_var[v], s)))
        tot += best
    return tot


def test_initial_lower_bound_matches_enumeration(tet_problem):
    inst, prob = tet_problem
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)
    o = S.DualOracle(dec)
    assert o.lower_bound() == pytest.approx(_lb0_brute(prob, dec), abs=1e-12)


@pytest.mark.parametrize("chunk", [0, 5])
def test_dual_invariants_tet(tet_problem, chunk):
    """sum_j l^j_i + |J_i| pend_i = c_i; pool bound non-decreasing every half-pass;
    E(l~) >= pool bound; LB <= LP* <= OPT (weak duality, Eq. D)."""
    inst, prob = tet_problem
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, chunk)
    o = S.DualOracle(dec)
    opt, x, nopt, _ = E.solve_exact(prob)
    lp = E.lp_relaxation(prob)
    prev = o.pool_bound()
    for t in range(60):
        for d in (+1, -1):
            o.half_pass(d)
            pb = o.pool_bound()
            assert pb >= prev - 1e-12 * max(1.0, abs(pb))
            prev = pb
            lb = o.lower_bound()
            assert lb >= pb - 1e-12
            assert lb <= opt + 1e-12
            if lp is not None:
                assert lb <= lp + 1e-12
        assert np.abs(o.feasibility_residual()).max() < 1e-12
    assert lp is None or lp <= opt + 1e-12


def test_dual_converges_to_lp_optimum_and_primal_is_optimal(tet_problem):
    inst, prob = tet_problem
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)
    o, trace = S.run_dual(dec, 100, lb_every=10)
    opt, x, nopt, nodes = E.solve_exact(prob)
    lp = E.lp_relaxation(prob)
    assert trace[-1][1] == pytest.approx(lp, rel=1e-9)
    res = PR.round_primal(o, prob, fixed)
    assert res.ok
    assert res.cost == pytest.approx(opt, abs=1e-12)
    assert not np.any(prob.residual(res.x))


def test_icosahedron_bound_primal_and_gap(ico_problem):
    inst, prob = ico_problem
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)
    o, trace = S.run_dual(dec, 200, lb_every=20)
    lbs = [t[1] for t in trace]
    assert all(b >= a - 1e-12 for a, b in zip(lbs, lbs[1:]))
    lp = E.lp_relaxation(prob)
    assert lbs[-1] <= lp + 1e-12
    res = PR.round_primal(o, prob, fixed)
    assert res.ok
    assert lbs[-1] <= res.cost + 1e-12
    # relative primal-dual gap (Sec. 4 "Optimality gaps")
    assert (res.cost - lbs[-1]) / res.cost < 1e-2
    # the recovered matching is the ground truth
    tt = (prob.vtype == P.TT) & (res.x == 1)
    assert np.all(inst.perm[prob.vm[tt]] == prob.vn[tt])
    assert tt.sum() == inst.X.nt


def test_zero_noise_copy_recovers_permutation():
    """Features copied exactly: OPT = 0 and only the relabelling attains it."""
    inst = I.tet(seed=3, feat_noise=0.0)
    prob, d, _ = P.make_problem(inst)
    opt, x, nopt, _ = E.solve_exact(prob)
    assert opt == pytest.approx(0.0, abs=1e-15) and nopt == 1
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)
    o, _ = S.run_dual(dec, 50)
    res = PR.round_primal(o, prob, fixed)
    assert res.ok and res.cost == pytest.approx(0.0, abs=1e-15)
    assert np.array_equal(res.x, x.astype(np.uint8))


def test_planted_mistakes_are_caught(tet_problem):
    """Each pin above fails when a plausible mistake is planted in the oracle."""
    inst, prob = tet_problem
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)
    # (a) wrong |J_i| in the averaging breaks dual feasibility
    o = S.DualOracle(dec)
    o.dec = B.Decomposition(**{**dec.__dict__, "deg": dec.deg + 1})
    o.iterate(3)
    assert np.abs(o.feasibility_residual()).max() > 1e-6
    # (b) a min-marginal with the wrong sign (lambda += omega M) lowers the bound
    o = S.DualOracle(dec, omega=-0.5)
    lb0 = o.pool_bound()
    o.iterate(5)
    assert o.pool_bound() < lb0 - 1e-9 or o.lower_bound() > E.lp_relaxation(prob) + 1e-9
    # (c) a flipped closedness sign on one element makes the ground truth infeasible
    bad = P.Problem(**{**prob.__dict__})
    bad.row_coef = prob.row_coef.copy()
    x = np.zeros(prob.nvars, np.int64)
    tt = np.nonzero(prob.vtype == P.TT)[0]
    hit = tt[np.all(inst.perm[prob.vm[tt]] == prob.vn[tt], axis=1)]
    x[hit] = 1
    pos = np.nonzero(bad.row_var[: bad.row_ptr[bad.n_closed]] == hit[0])[0][0]
    bad.row_coef[pos] *= -1
    assert np.any(bad.residual(x))
