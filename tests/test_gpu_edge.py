"""Degenerate cases on the GPU path: a pair whose presolve fixes every variable (an empty BDD
store: the bound is the presolve constant, the matching is the fixed one), the same pair in a
batch beside a normal one, and zero dual iterations (bound and gradient at lambda^0 against
the FP64 oracle)."""
import numpy as np
import pytest

from oracle import bdd as B
from oracle import grad as G
from oracle import problem as P
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


def _fully_fixed():
    inst = I.tet()
    d = P.pair_distance(inst.FX, inst.FY).astype(np.float32)
    al = np.zeros(d.shape, np.uint8)
    al[np.arange(inst.X.nv), inst.perm] = 1
    prob = P.build_problem(inst.X.T, inst.Y.T, d.astype(np.float64), al.astype(bool), normalize=False)
    fixed, const = P.presolve(prob)
    assert np.all(fixed >= 0)
    return inst, d, al, prob, fixed, const


def test_empty_store(torch):
    from paper_2310_08230_gb300.api import Solver

    inst, d, al, prob, fixed, const = _fully_fixed()
    s = Solver(inst.X.T, inst.Y.T, d, al, normalize_costs=0)
    info = s.info()
    assert info["nvars_free"] == 0 and info["nslots"] == 0
    s.dual(5)
    s.dual_qn(2, 3)
    assert s.lower_bound() == pytest.approx(const, rel=1e-12)
    n, lb, ok = s.converge(100)
    assert ok and lb == pytest.approx(const, rel=1e-12)
    x, cost, ok = s.primal()
    assert ok and np.array_equal(x, (fixed == 1).astype(np.uint8))
    assert cost == pytest.approx(const, rel=1e-12)
    s.record(4, 2)
    g = s.grad().reshape(d.shape)
    # the bound is the sum of the fixed elements' mean pair costs; every vertex of the
    # tetrahedron is a corner of three matched triangles, so each matched pair has gradient 1
    assert np.all(g[al == 0] == 0)
    np.testing.assert_allclose(g[al == 1], 1.0, rtol=1e-6)
    s.close()


def test_empty_instance_in_a_batch(torch):
    from paper_2310_08230_gb300.api import Solver

    inst, d, al, prob, fixed, const = _fully_fixed()
    other = I.config1()
    p2, d2, _ = P.make_problem(other)
    b = Solver.batch([(inst.X.T, inst.Y.T, d, al), (other.X.T, other.Y.T, d2.astype(np.float32), None)],
                     normalize_costs=0)
    one = Solver(other.X.T, other.Y.T, d2.astype(np.float32), None, normalize_costs=0)
    b.dual(20)
    one.dual(20)
    lbs = b.lower_bounds()
    assert lbs[0] == pytest.approx(const, rel=1e-12)
    assert lbs[1] == pytest.approx(one.lower_bound(), rel=1e-12)
    xs, costs, ok = b.primal_batch()
    assert ok.all() and np.array_equal(xs[0], (fixed == 1).astype(np.uint8))
    b.close()
    one.close()


def test_zero_iterations_bound_and_gradient(torch):
    from paper_2310_08230_gb300.api import Solver

    inst = I.tet()
    prob, d, _ = P.make_problem(inst)
    d32 = d.astype(np.float32)
    s = Solver(inst.X.T, inst.Y.T, d32, None, normalize_costs=0)
    s.record(0, 1)
    lb = s.lower_bound()
    g = s.grad().reshape(d.shape)
    prob = P.build_problem(inst.X.T, inst.Y.T, d32.astype(np.float64), None, normalize=False)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)
    ref_lb, gc = G.bound_and_grad(dec, prob.cost, fixed, 0)
    assert lb == pytest.approx(ref_lb, rel=1e-5)
    ref = np.zeros(d.shape)
    for v in range(3):
        np.add.at(ref, (prob.vm[:, v], prob.vn[:, v]), gc / 3.0)
    assert np.linalg.norm(g - ref) <= 1e-4 * np.linalg.norm(ref)
    s.close()
