"""Eq. 2 costs on the GPU path (cost_model = 1: mixed-area-weighted feature distances)
against the FP64 oracle: pair distances to 1e-5 relative, the bound after a fixed number of
iterations to 1e-5 relative, and a feasible primal whose cost is recomputed exactly."""
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


def test_pair_distances_match_oracle(torch):
    from paper_2310_08230_gb300.api import pair_distances

    inst = I.config2()
    d = pair_distances(torch.from_numpy(inst.FX).cuda(), torch.from_numpy(inst.FY).cuda()).cpu().numpy()
    ref = P.pair_euclid(inst.FX, inst.FY)
    np.testing.assert_allclose(d, ref, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("which,chunk,iters", [("tet", 0, 40), ("config1", 0, 30), ("config2", 16, 30)])
def test_eq2_bound_and_primal(torch, which, chunk, iters):
    from paper_2310_08230_gb300.api import Solver

    inst = getattr(I, which)()
    _, _, allowed = P.make_problem(inst)
    al = None if inst.topk is None else allowed
    d = P.pair_euclid(inst.FX, inst.FY).astype(np.float32)
    prob = P.build_problem(inst.X.T, inst.Y.T, d.astype(np.float64), al, cost_model=1, VX=inst.X.V, VY=inst.Y.V)
    fixed, const = P.presolve(prob)
    o = S.DualOracle(B.decompose(prob, fixed, const, chunk))
    o.iterate(iters)
    ref = o.lower_bound()
    s = Solver(inst.X.T, inst.Y.T, d, al, VX=inst.X.V, VY=inst.Y.V, cost_model=1, split_chunk=chunk)
    s.dual(iters)
    lb = s.lower_bound()
    assert abs(lb - ref) <= 1e-5 * max(abs(ref), 1e-3)
    x, cost, ok = s.primal()
    assert ok and not np.any(prob.residual(x))
    assert cost == pytest.approx(float(prob.cost @ x), rel=1e-6)
    assert lb <= cost + 1e-5 * abs(cost)  # the bound's tolerance: 1e-5 relative (FP32 min-sum)
    s.close()


def test_eq2_needs_positions(torch):
    from paper_2310_08230_gb300 import _lib as L
    from paper_2310_08230_gb300.api import Solver

    inst = I.tet()
    d = P.pair_euclid(inst.FX, inst.FY).astype(np.float32)
    with pytest.raises(L.DiscoError):
        Solver(inst.X.T, inst.Y.T, d, None, cost_model=1)


@pytest.mark.parametrize("normalize", [0, 1])
def test_eq2_gradient_matches_fp64_autograd(torch, normalize):
    """The gradient through Eq. 2 costs: the FP64 replica's element-cost gradient, chained to
    the pair distances with each corner's weight A_X(m) + A_Y(n)."""
    from oracle import grad as G
    from paper_2310_08230_gb300.api import Solver

    inst = I.tet()
    d = P.pair_euclid(inst.FX, inst.FY).astype(np.float32)
    iters, every = 12, 5
    s = Solver(inst.X.T, inst.Y.T, d, None, VX=inst.X.V, VY=inst.Y.V, cost_model=1, normalize_costs=normalize,
               graph_iters=0)
    s.record(iters, every)
    g = s.grad().reshape(d.shape)
    s.close()
    prob = P.build_problem(inst.X.T, inst.Y.T, d.astype(np.float64), None, cost_model=1, VX=inst.X.V, VY=inst.Y.V,
                           normalize=False)
    fixed, const = P.presolve(prob)
    raw = prob.cost.copy()
    scale = raw.max() if normalize else 1.0
    c = raw / scale
    _, gc = G.bound_and_grad(B.decompose(prob, fixed, const / scale, 0), c, fixed, iters)
    graw = gc / scale
    if normalize:
        graw[int(np.argmax(raw))] -= float(gc @ c) / scale
    aX, aY = P.mixed_areas(inst.X.V, inst.X.T), P.mixed_areas(inst.Y.V, inst.Y.T)
    ref = np.zeros(d.shape)
    for v in range(3):
        np.add.at(ref, (prob.vm[:, v], prob.vn[:, v]), graw * (aX[prob.vm[:, v]] + aY[prob.vn[:, v]]))
    err = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
    assert err < 1e-3, err
