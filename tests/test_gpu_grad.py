"""Gradient of the dual bound w.r.t. the pair costs (disco_record / disco_grad, adjoint
kernels) against the FP64 autograd replica of the same unrolled iterations
(``oracle/grad.py``, itself pinned to the C oracle and to finite differences) and against
central differences of the GPU bound.

Tolerances: the gradient to 1e-3 in relative 2-norm (FP32 adjoints of O(10^5) min-plus
steps; a mismatched tie would show up as an O(1) error); the bound to 1e-5 relative to the
larger of itself and the largest element cost (raw costs are not scaled to [0, 1]);
directional finite differences (eps 1e-3) to 2 % of the directional derivative's scale."""
import numpy as np
import pytest

from oracle import bdd as B
from oracle import grad as G
from oracle import problem as P
from synth import instances as I
from synth import meshes as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08230_gb300.build import build

    build()
    return torch


def _small_topk(k=6):
    rng = np.random.Generator(np.random.PCG64(5))
    X = M.icosphere(1)
    Y, FX, FY, perm = I.make_pair(X, rng, 16, 0.05, deform=True)
    return I.Instance(f"icosphere1-80T-top{k}", X, Y, FX, FY, perm, k, 30)


def _case(name):
    return _small_topk(3) if name == "ico1" else getattr(I, name)()


def _oracle_pair_grad(inst, d, allowed, chunk, iters, normalize):
    """Bound and d bound / d pair costs from the FP64 replica, chained like the library."""
    prob = P.build_problem(inst.X.T, inst.Y.T, d.astype(np.float64), allowed)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, chunk)
    raw = d.astype(np.float64)[prob.vm, prob.vn].mean(axis=1)
    scale = raw.max() if normalize else 1.0
    c = raw / scale
    lb, gc = G.bound_and_grad(dec, c, fixed, iters)
    graw = gc / scale
    if normalize:
        graw[int(np.argmax(raw))] -= float(gc @ c) / scale
    gp = np.zeros(d.shape)
    for v in range(3):
        np.add.at(gp, (prob.vm[:, v], prob.vn[:, v]), graw / 3.0)
    return lb, gp, float(c.max())


def _solver(inst, d, allowed, **kw):
    from paper_2310_08230_gb300.api import Solver

    return Solver(inst.X.T, inst.Y.T, np.asarray(d, np.float32), allowed, **kw)


@pytest.mark.parametrize("name,chunk,iters,every,normalize",
                         [("tet", 0, 30, 7, 0), ("tet", 3, 20, 20, 1), ("config1", 4, 10, 4, 0),
                          ("ico1", 6, 8, 3, 0), ("ico1", 6, 6, 4, 1)])
def test_grad_matches_fp64_autograd(torch, name, chunk, iters, every, normalize):
    inst = _case(name)
    prob, d, allowed = P.make_problem(inst)
    al = None if inst.topk is None else allowed
    d32 = d.astype(np.float32)
    s = _solver(inst, d32, al, split_chunk=chunk, normalize_costs=normalize, graph_iters=0)
    s.record(iters, every)
    lb = s.lower_bound()
    g = s.grad().reshape(d.shape)
    ref_lb, ref_g, cmax = _oracle_pair_grad(inst, d32, al, chunk, iters, normalize)
    # FP32 error relative to the cost scale (the bound is a cancelling sum of costs)
    assert abs(lb - ref_lb) <= 1e-5 * max(abs(ref_lb), cmax)
    err = np.linalg.norm(g - ref_g) / max(np.linalg.norm(ref_g), 1e-30)
    assert err < 1e-3, err
    s.close()


def test_grad_matches_gpu_finite_differences(torch):
    inst = _small_topk()
    prob, d, allowed = P.make_problem(inst)
    d32 = d.astype(np.float32)
    iters, eps = 20, 1e-3
    s = _solver(inst, d32, allowed, normalize_costs=0)
    s.record(iters, 10)
    g = s.grad().reshape(d.shape)
    s.close()
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = (rng.standard_normal(d.shape) * allowed).astype(np.float32)
        vals = []
        for sgn in (1, -1):
            t = _solver(inst, d32 + sgn * eps * v, allowed, normalize_costs=0)
            t.record(iters, 10)
            vals.append(t.lower_bound())
            t.close()
        fd = (vals[0] - vals[1]) / (2 * eps)
        dd = float((g.astype(np.float64) * v).sum())
        scale = float(np.abs(g).sum() * np.abs(v).max())
        assert abs(fd - dd) <= 0.02 * scale, (fd, dd, scale)


def test_grad_keeps_state_and_repeats(torch):
    inst = I.tet()
    prob, d, allowed = P.make_problem(inst)
    s = _solver(inst, d.astype(np.float32), None)
    s.record(15, 4)
    lam0, pend0 = s.get_state()
    lb0 = s.lower_bound()
    g1 = s.grad()
    g2 = s.grad()
    lam1, pend1 = s.get_state()
    np.testing.assert_array_equal(g1, g2)
    np.testing.assert_array_equal(lam0, lam1)
    np.testing.assert_array_equal(pend0, pend1)
    assert s.lower_bound() == lb0
    s.dual(5)  # the handle keeps working after a gradient
    assert s.info()["iterations"] == 20
    s.close()


def test_autograd_function_matches_solver(torch):
    from paper_2310_08230_gb300.autograd import dual_bounds

    insts = [I.tet(), _small_topk()]
    costs, meshes, masks, refs = [], [], [], []
    for inst in insts:
        prob, d, allowed = P.make_problem(inst)
        al = None if inst.topk is None else allowed
        s = _solver(inst, d.astype(np.float32), al, normalize_costs=0)
        s.record(12, 5)
        refs.append((s.lower_bound(), s.grad().reshape(d.shape)))
        s.close()
        costs.append(torch.tensor(d.astype(np.float32), device="cuda", requires_grad=True))
        meshes.append((inst.X.T, inst.Y.T))
        masks.append(None if al is None else torch.tensor(al.astype(np.uint8), device="cuda"))
    lbs = dual_bounds(costs, meshes, masks, iters=12, checkpoint_every=5, normalize_costs=0)
    w = torch.tensor([2.0, -0.5], dtype=torch.float64, device="cuda")
    (lbs * w).sum().backward()
    for k, (lb, g) in enumerate(refs):
        assert float(lbs[k].detach()) == pytest.approx(lb, rel=1e-12)
        np.testing.assert_allclose(costs[k].grad.cpu().numpy(), float(w[k]) * g, rtol=1e-6, atol=1e-12)
