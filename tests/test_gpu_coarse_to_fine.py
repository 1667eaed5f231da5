"""Coarse-to-fine solving on the GPU path: a coarse solve, its point map (equal to the
oracle's point map of the same matching), a fine candidate mask one ring around it, and a
fine solve whose bound matches the oracle's on the same mask (1e-5 relative) and whose
matching is feasible and close to the ground truth."""
import numpy as np
import pytest

from oracle import bdd as B
from oracle import problem as P
from oracle import solver as S
from synth import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08230_gb300.build import build

    build()
    return torch


def test_coarse_to_fine(torch):
    from paper_2310_08230_gb300.api import Solver, candidates_coarse_to_fine

    coarse, fine, cx, cy = I.coarse_fine_pair(2)
    dc = P.pair_distance(coarse.FX, coarse.FY).astype(np.float32)
    sc = Solver(coarse.X.T, coarse.Y.T, dc, None)
    sc.dual(100)
    xc, cost_c, ok = sc.primal()
    assert ok
    pairs = sc.point_map(xc)
    prob_c = P.build_problem(coarse.X.T, coarse.Y.T, dc.astype(np.float64), None)
    np.testing.assert_array_equal(pairs, P.point_map(prob_c, xc))
    sc.close()
    allowed = candidates_coarse_to_fine(pairs, cx, cy, 1, fine.X.T, fine.X.nv, fine.Y.T, fine.Y.nv)
    df = P.pair_distance(fine.FX, fine.FY).astype(np.float32)
    sf = Solver(fine.X.T, fine.Y.T, df, allowed)
    sf.dual(60)
    lb = sf.lower_bound()
    prob_f = P.build_problem(fine.X.T, fine.Y.T, df.astype(np.float64), allowed.astype(bool))
    fixed, const = P.presolve(prob_f)
    o = S.DualOracle(B.decompose(prob_f, fixed, const, 0))
    o.iterate(60)
    assert abs(lb - o.lower_bound()) <= 1e-5 * max(abs(o.lower_bound()), 1e-3)
    xf, cost_f, okf = sf.primal()
    assert okf and not np.any(prob_f.residual(xf))
    pf = sf.point_map(xf)
    hits = np.mean(fine.perm[pf[:, 0]] == pf[:, 1])
    assert hits > 0.9, hits
    sf.close()


def test_three_levels(torch):
    """80 -> 320 -> 1280 triangles, one ring of candidates around each level's matching:
    every level's matching is feasible, the finest recovers the ground truth on most
    vertices, and it is solved on a small fraction of its product space."""
    from paper_2310_08230_gb300.api import solve_coarse_to_fine

    levels = I.multilevel_pair()
    costs = [P.pair_distance(inst.FX, inst.FY).astype(np.float32) for inst, _, _ in levels]
    res = solve_coarse_to_fine([(inst.X.T, inst.Y.T, cx, cy) for inst, cx, cy in levels], costs, rings=1, iters=80)
    assert len(res) == 3 and all(r["feasible"] for r in res)
    fine = levels[-1][0]
    pf = res[-1]["pairs"]
    assert np.mean(fine.perm[pf[:, 0]] == pf[:, 1]) > 0.9
    assert res[-1]["density"] < 0.05
    # bound <= feasible cost, to the bound's own tolerance (1e-5 relative, FP32 min-sum)
    assert all(r["lower_bound"] <= r["cost"] + 1e-5 * abs(r["cost"]) for r in res)
