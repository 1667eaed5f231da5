"""Gradient of the dual bound w.r.t. the pair costs (disco_record / disco_grad, adjoint
kernels) against the FP64 autograd replica of the same unrolled iterations
(``oracle/grad.py``, itself pinned to the C oracle and to finite differences) and against
central differences of the GPU bound, and at the differentiated workload's size through the
feature MLP against the replica chained through the same MLP in FP64.

Tolerances: the gradient to 1e-3 in relative 2-norm (FP32 adjoints of O(10^5) min-plus
steps; a mismatched tie would show up as an O(1) error); the bound to 1e-5 relative to the
larger of itself and the largest element cost (raw costs are not scaled to [0, 1]);
directional finite differences (eps 1e-3) to 2 % of the directional derivative's scale."""
import numpy as np
import pytest
import torch as T

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


def test_mlp_parameter_gradient_at_full_scale(torch):
    """The differentiated workload at its size: one 1280-triangle icosphere pair, raw 128-d
    features through the 128-256-64 ReLU MLP, costs = squared distances of the MLP outputs
    (not normalised), top-16 candidates held fixed. d(bound after 10 iterations) / d(MLP
    parameters) from the adjoint kernels, through dual_bounds and the MLP in FP32 on the
    GPU, against the FP64 replica chained through the same MLP in FP64 on the CPU, to 1e-3
    in relative 2-norm. Both solvers receive the same FP32 costs (the FP64 MLP's, rounded);
    on the GPU a straight-through identity passes them in while the gradient flows back
    through the FP32 MLP."""
    from paper_2310_08230_gb300.autograd import dual_bounds

    iters, every = 10, 4
    inst = I.config5(1)[0]
    raw = I.mlp_params()
    # FP64 reference: costs, the replica's gradient w.r.t. them, chained to the parameters
    ps64 = [T.tensor(p, dtype=T.float64, requires_grad=True) for p in raw]

    def mlp(F, ps):
        W1, b1, W2, b2 = ps
        return T.relu(F @ W1.T + b1) @ W2.T + b2

    a = mlp(T.tensor(inst.FX, dtype=T.float64), ps64)
    b = mlp(T.tensor(inst.FY, dtype=T.float64), ps64)
    d64 = ((a[:, None, :] - b[None, :, :]) ** 2).sum(-1)
    d32 = d64.detach().numpy().astype(np.float32)
    allowed = P.candidate_pairs(d32.astype(np.float64), inst.topk, inst.X.T, inst.Y.T)
    ref_lb, gd, _ = _oracle_pair_grad(inst, d32, allowed, 0, iters, False)
    ref = T.autograd.grad(d64, ps64, grad_outputs=T.tensor(gd))
    # GPU: MLP in FP32, solver on the same FP32 costs, adjoint back to the parameters
    ps = [torch.tensor(p, device="cuda", requires_grad=True) for p in raw]
    FX = torch.from_numpy(inst.FX).cuda()
    FY = torch.from_numpy(inst.FY).cuda()
    W1, b1, W2, b2 = ps
    ga = torch.relu(FX @ W1.T + b1) @ W2.T + b2
    gb = torch.relu(FY @ W1.T + b1) @ W2.T + b2
    dg = ((ga[:, None, :] - gb[None, :, :]) ** 2).sum(-1)
    d_in = dg + (torch.from_numpy(d32).cuda() - dg).detach()  # value d32, gradient into dg
    mask = torch.from_numpy(allowed.astype(np.uint8)).cuda()
    lbs = dual_bounds([d_in], [(inst.X.T, inst.Y.T)], [mask], iters, every, normalize_costs=0)
    lbs.sum().backward()
    assert abs(float(lbs[0].detach()) - ref_lb) <= 1e-5 * abs(ref_lb)
    got = np.concatenate([p.grad.detach().cpu().numpy().ravel() for p in ps])
    want = np.concatenate([r.numpy().ravel() for r in ref])
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-3, err


def test_adjoint_matches_fp64_central_differences_at_full_scale(torch):
    """d(bound after 50 iterations) / d(pair costs) of the differentiated workload's first pair
    (the adjoint kernels, checkpoint every 10) along three random directions, against central
    differences of the FP64 C oracle's bound at eps 1e-6: FP64 leaves no rounding floor at
    that step, and at a generic point it crosses no kink of the piecewise-linear bound. The
    presolve depends only on feasibility, so one decomposition serves every perturbed cost
    vector; each side is agreed to 1e-3 of the directional derivative's scale."""
    import dataclasses

    from oracle import solver as S
    from paper_2310_08230_gb300.api import Solver

    iters, every, eps = 50, 10, 1e-6
    inst = I.config5(1)[0]
    W1, b1, W2, b2 = [p.astype(np.float64) for p in I.mlp_params()]
    fa = np.maximum(inst.FX.astype(np.float64) @ W1.T + b1, 0.0) @ W2.T + b2
    fb = np.maximum(inst.FY.astype(np.float64) @ W1.T + b1, 0.0) @ W2.T + b2
    d32 = ((fa[:, None, :] - fb[None, :, :]) ** 2).sum(-1).astype(np.float32)
    allowed = P.candidate_pairs(d32.astype(np.float64), inst.topk, inst.X.T, inst.Y.T)
    prob = P.build_problem(inst.X.T, inst.Y.T, d32.astype(np.float64), allowed, normalize=False)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)

    def oracle_bound(dd):
        c = dd[prob.vm, prob.vn].mean(axis=1)
        cost = np.concatenate([c, np.zeros(dec.nvars_total - dec.nvars)])
        o = S.DualOracle(dataclasses.replace(dec, cost=cost, const=float(c[fixed == 1].sum())))
        o.iterate(iters)
        return o.lower_bound()

    s = Solver(inst.X.T, inst.Y.T, d32, allowed.astype(np.uint8), normalize_costs=0)
    s.record(iters, every)
    g = s.grad().reshape(d32.shape).astype(np.float64)
    lb = s.lower_bound()
    s.close()
    base = d32.astype(np.float64)
    assert abs(lb - oracle_bound(base)) <= 1e-5 * abs(lb)
    rng = np.random.default_rng(17)
    for _ in range(3):
        v = rng.standard_normal(d32.shape) * allowed
        fd = (oracle_bound(base + eps * v) - oracle_bound(base - eps * v)) / (2 * eps)
        dd = float((g * v).sum())
        scale = float(np.abs(g * v).sum())
        assert abs(fd - dd) <= 1e-3 * scale, (fd, dd, scale)
