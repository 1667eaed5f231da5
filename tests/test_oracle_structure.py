"""Pins of the oracle's problem construction and BDD compiler (CPU only).

Product space (Sec. 3.1, Fig. 2), constraints (Eq. P), BDDs and splitting
(App. A.3, Alg. 3, Fig. BDD)."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import bdd as B
from oracle import problem as P
from synth import instances as I
from synth import meshes as M

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _counts(TX, TY, nvx, nvy):
    tx, ty = len(TX), len(TY)
    ex, ey = len(P.mesh_edges(TX)), len(P.mesh_edges(TY))
    return tx, ty, ex, ey, nvx, nvy


@pytest.mark.parametrize("mk", [M.tetrahedron, M.icosahedron, lambda: M.icosphere(1), lambda: M.torus(4, 5)])
def test_meshes_closed_oriented(mk):
    m = mk()
    chi = P.check_mesh(m.nv, m.T)
    assert chi in (2, 0)


def test_mesh_checks_reject_bad_meshes():
    m = M.icosahedron()
    with pytest.raises(ValueError):  # one flipped triangle
        T = m.T.copy()
        T[0] = T[0][[0, 2, 1]]
        P.check_mesh(m.nv, T)
    with pytest.raises(ValueError):  # open mesh
        P.check_mesh(m.nv, m.T[1:])


@pytest.mark.parametrize("which", ["tet", "ico", "torus"])
def test_product_space_counts_closed_form(which):
    """|P| = 3TT' + 6(TE' + T'E) + TV' + T'V for the full product space; each element
    lies in exactly 3 closedness rows; tri-tri elements in 2 projection rows, the others
    in 1; closedness rows = 2EE' + EV' + VE' (Sec. 3.1; ~21-22 |T||T'|, App. B)."""
    if which == "tet":
        X = M.tetrahedron()
    elif which == "ico":
        X = M.icosahedron()
    else:
        X = M.torus(3, 4)
    rng = np.random.Generator(np.random.PCG64(5))
    Y, _ = M.relabel(X, rng)
    d = np.ones((X.nv, Y.nv))
    prob = P.build_problem(X.T, Y.T, d)
    tx, ty, ex, ey, vx, vy = _counts(X.T, Y.T, X.nv, Y.nv)
    assert prob.nvars == 3 * tx * ty + 6 * (tx * ey + ty * ex) + tx * vy + ty * vx
    assert prob.n_closed == 2 * ex * ey + ex * vy + vx * ey
    assert prob.n_projx == tx and prob.n_projy == ty
    per_var = np.bincount(prob.row_var[: prob.row_ptr[prob.n_closed]], minlength=prob.nvars)
    assert np.all(per_var == 3)
    proj = np.bincount(prob.row_var[prob.row_ptr[prob.n_closed]:], minlength=prob.nvars)
    assert np.all(proj[prob.vtype == P.TT] == 2)
    assert np.all(proj[prob.vtype != P.TT] == 1)
    ratio = prob.nvars / (tx * ty)
    if which == "ico":
        assert 21.0 <= ratio <= 23.0
    if which == "tet":
        assert prob.nvars == 368


def _gt_solution(prob, inst):
    """Indicator of the ground-truth matching: tri-tri elements t -> perm(t) with matching rotation."""
    x = np.zeros(prob.nvars, np.int64)
    tt = np.nonzero(prob.vtype == P.TT)[0]
    mapped = inst.perm[prob.vm[tt]]
    hit = np.all(mapped == prob.vn[tt], axis=1)
    x[tt[hit]] = 1
    return x


@pytest.mark.parametrize("mk", [I.tet, I.config1, I.config2])
def test_ground_truth_matching_is_feasible(mk):
    """The relabelled identity satisfies every row exactly: pins orientation, rotation
    enumeration and the sign convention of the closedness rows (Eq. P)."""
    inst = mk()
    prob, _, _ = P.make_problem(inst)
    x = _gt_solution(prob, inst)
    assert x.sum() == inst.X.nt
    assert not np.any(prob.residual(x))


def test_ground_truth_torus_feasible():
    rng = np.random.Generator(np.random.PCG64(11))
    X = M.torus(4, 5)
    Y, FX, FY, perm = I.make_pair(X, rng, 8, 0.05, deform=True)
    inst = I.Instance("torus", X, Y, FX, FY, perm, None, 10)
    prob, _, _ = P.make_problem(inst)
    x = _gt_solution(prob, inst)
    assert not np.any(prob.residual(x))
    # a wrong rotation of one triangle breaks closedness
    tt = np.nonzero(x)[0][0]
    same = np.nonzero((prob.vtype == P.TT) & (prob.vx == prob.vx[tt]) & (prob.vy == prob.vy[tt]))[0]
    x2 = x.copy()
    x2[tt] = 0
    x2[[v for v in same if v != tt][0]] = 1
    assert np.any(prob.residual(x2)[: prob.n_closed])


def test_pruned_space_keeps_ground_truth_and_presolve_keeps_it_feasible():
    inst = I.config2()
    prob, d, allowed = P.make_problem(inst)
    assert np.all(allowed[np.arange(inst.X.nv), inst.perm])
    fixed, const = P.presolve(prob)
    x = _gt_solution(prob, inst)
    # presolve only fixes variables every feasible solution agrees on
    assert np.all(x[fixed == 1] == 1) and np.all(x[fixed == 0] == 0)


def test_presolve_fixpoint_matches_brute_force_on_small_rows():
    """GAC of a single +-1 row equals the brute-force support of each variable."""
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(200):
        n = int(rng.integers(1, 7))
        coef = rng.choice([-1, 1], n)
        rhs = int(rng.integers(-2, 3))
        prob = P.Problem(1, 1, np.zeros((n, 3), np.int64), np.zeros((n, 3), np.int64), np.zeros(n, np.int64),
                         np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n),
                         np.array([0, n]), np.arange(n), coef, np.array([rhs]), 1, 0, 0, np.array([0]))
        sols = [s for s in itertools.product([0, 1], repeat=n) if np.dot(coef, s) == rhs]
        if not sols:
            with pytest.raises(P.Infeasible):
                P.gac(prob, -np.ones(n, np.int8))
            continue
        fixed = P.gac(prob, -np.ones(n, np.int8))
        S = np.array(sols)
        for i in range(n):
            vals = set(S[:, i])
            if vals == {0}:
                assert fixed[i] == 0
            elif vals == {1}:
                assert fixed[i] == 1
            else:
                assert fixed[i] == -1


# ---------------------------------------------------------------- BDDs ------------
def test_fig_bdd_widths_and_split():
    g = json.load(open(os.path.join(GOLD, "fig_bdd.json")))
    n = g["row"]["n"]
    bdd, _ = B.compile_row(np.arange(n), np.ones(n, np.int64), g["row"]["rhs"])
    assert bdd.widths() == g["widths"]
    assert bdd.n_nodes() == g["n_nodes"]
    segs, aux, nxt = B.split_row(bdd, g["split_chunk"], 100)
    assert len(segs) == 2 and aux == [100, 101, 102]
    left, right = segs
    assert left.widths() == g["left"]["widths"]
    assert right.widths() == g["right"]["widths"]
    assert left.var == [0, 1, 2, 3, 100, 101, 102]
    assert right.var == [100, 101, 102, 4, 5, 6, 7]


@pytest.mark.parametrize("seed", range(6))
def test_bdd_accepts_exactly_the_row_solutions(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(30):
        n = int(rng.integers(2, 10))
        coef = rng.choice([-1, 1], n)
        sols = set()
        for s in itertools.product([0, 1], repeat=n):
            sols.add(int(np.dot(coef, s)))
        rhs = int(rng.choice(sorted(sols)))
        bdd, _ = B.compile_row(np.arange(n), coef, rhs)
        assert bdd.widths()[0] == 1
        for s in itertools.product([0, 1], repeat=n):
            assert bdd.evaluate(dict(enumerate(s))) == (np.dot(coef, s) == rhs)
        # reduced: no two nodes of a layer with the same children
        for l in range(n):
            pairs = list(zip(bdd.lo[l], bdd.hi[l]))
            assert len(set(pairs)) == len(pairs)
            assert all(p != (B.BOT, B.BOT) for p in pairs)


@pytest.mark.parametrize("chunk", [2, 3, 4, 5])
def test_split_segments_are_equivalent_to_the_row(chunk):
    """Alg. 3: the sub-BDDs together accept exactly the row's solutions, and the
    one-hot auxiliaries are determined by x (y_j = 1 iff node j of the cut layer is used)."""
    rng = np.random.Generator(np.random.PCG64(chunk))
    for _ in range(20):
        n = int(rng.integers(3, 10))
        coef = rng.choice([-1, 1], n)
        vals = {int(np.dot(coef, s)) for s in itertools.product([0, 1], repeat=n)}
        rhs = int(rng.choice(sorted(vals)))
        bdd, sums = B.compile_row(np.arange(n), coef, rhs)
        segs, aux, _ = B.split_row(bdd, chunk, n)
        if len(aux) > 10:
            continue
        for s in itertools.product([0, 1], repeat=n):
            feas = np.dot(coef, s) == rhs
            good = 0
            for y in itertools.product([0, 1], repeat=len(aux)):
                a = dict(enumerate(s))
                a.update(zip(aux, y))
                if all(seg.evaluate(a) for seg in segs):
                    good += 1
            assert good == (1 if feas else 0)


def test_decompose_problem_rows():
    inst = I.tet()
    prob, _, _ = P.make_problem(inst)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)
    assert dec.nb == prob.nrows
    assert np.all(dec.deg[: prob.nvars][prob.vtype == P.TT] == 5)
    assert np.all(dec.deg[: prob.nvars][prob.vtype != P.TT] == 4)
    dec4 = B.decompose(prob, fixed, const, 4)
    assert dec4.nb > dec.nb
    assert np.all(dec4.deg[prob.nvars:] == 2)
    assert np.array_equal(dec4.deg[: prob.nvars], dec.deg[: prob.nvars])
