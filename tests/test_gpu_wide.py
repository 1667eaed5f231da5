"""The width-16 and width-32 kernels, and Alg. 3's splitting without a segment cap, against
the FP64 oracle.

The icosphere workloads never have a BDD layer wider than 8 nodes. The bipyramid pairs
(two apexes of valence n over an n-gon, full product space) have long closedness rows around
the apexes: n = 12 gives layers up to 14 nodes wide, n = 16 up to 18, so their segments run
in the width-16 and width-32 kernels (forward / backward half-passes, bound, min-marginals,
rounding passes and adjoints) beside the fused 2/4/6 and the width-8 ones.

``split_max_segments = 0`` cuts every row into ceil(layers / chunk) segments, the literal
chunking of App. A.3 (Alg. 3); the library's default caps it at 8 segments per row.

Tolerances as in ``test_gpu_parity.py`` and ``test_gpu_grad.py``."""
import numpy as np
import pytest

from oracle import bdd as B
from oracle import grad as G
from oracle import primal as PR
from oracle import problem as P
from oracle import solver as S
from synth import instances as I

pytestmark = pytest.mark.gpu

LB_RTOL = 1e-5
MM_ATOL = 1e-4


@pytest.fixture(scope="module")
def torch():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08230_gb300.build import build

    build()
    return torch


def _launch_groups(dec) -> int:
    """Launches per pass over the device store: a segment goes to the narrowest width class
    (2, 4, 6, 8, 16, 32) that holds its widest layer; classes 2, 4 and 6 share one launch."""
    w = np.diff(dec.layer_node_ptr)
    seg_w = np.maximum.reduceat(w, dec.bdd_layer_ptr[:-1])
    return len({0 if x <= 6 else 8 if x <= 8 else 16 if x <= 16 else 32 for x in seg_w})


def _problem(inst, chunk, maxseg=8):
    prob, d, allowed = P.make_problem(inst)
    fixed, const = P.presolve(prob)
    return prob, d, allowed, fixed, const, B.decompose(prob, fixed, const, chunk, maxseg)


def _solver(inst, d, allowed=None, **kw):
    from paper_2310_08230_gb300.api import Solver

    return Solver(inst.X.T, inst.Y.T, np.asarray(d, np.float32), allowed, **kw)


@pytest.mark.parametrize("n,chunk,iters", [(12, 0, 60), (16, 0, 60), (16, 32, 40)])
def test_wide_classes_bound_min_marginals_and_primal(torch, n, chunk, iters):
    from paper_2310_08230_gb300 import _lib as L

    inst = I.bipyramid_pair(n)
    prob, d, allowed, fixed, const, dec = _problem(inst, chunk)
    w = np.diff(dec.layer_node_ptr)
    assert w.max() > (8 if n == 12 else 16)  # n = 12: the width-16 class; n = 16: the width-32 one
    s = _solver(inst, d, split_chunk=chunk, graph_iters=0, autotune=0)
    assert s.info()["max_width"] == w.max()
    # one launch per group and pass: the initial backward pass and the two half-passes of
    # the first iteration, no graph
    groups = _launch_groups(dec)
    assert groups >= 2  # the fused 2 / 4 / 6 launch and the wide class
    n0 = L.lib().disco_kernel_launches()
    s.dual(1)
    assert L.lib().disco_kernel_launches() - n0 == 3 * groups
    s.dual(iters - 1)
    o = S.DualOracle(dec)
    o.iterate(iters)
    lb, ref = s.lower_bound(), o.lower_bound()
    assert abs(lb - ref) <= LB_RTOL * max(abs(ref), 1e-3), (lb, ref)
    np.testing.assert_allclose(s.min_marginals(), o.min_marginals(), atol=MM_ATOL, rtol=0)
    x, cost, ok = s.primal()
    r = PR.round_primal(o, prob, fixed)
    assert ok and r.ok and not np.any(prob.residual(x))
    assert abs(cost - r.cost) <= 1e-4 * max(abs(r.cost), 1e-12), (cost, r.cost)
    s.close()


@pytest.mark.parametrize("n", [12, 16])
def test_wide_classes_gradient_matches_fp64_replica(torch, n):
    inst = I.bipyramid_pair(n)
    prob, d, allowed, fixed, const, dec = _problem(inst, 0)
    d32 = d.astype(np.float32)
    s = _solver(inst, d32, normalize_costs=0, graph_iters=0)
    s.record(8, 3)
    g = s.grad().reshape(d.shape)
    raw = d32.astype(np.float64)[prob.vm, prob.vn].mean(axis=1)
    lb_ref, gc = G.bound_and_grad(dec, raw, fixed, 8)
    gref = np.zeros(d.shape)
    for v in range(3):
        np.add.at(gref, (prob.vm[:, v], prob.vn[:, v]), gc / 3.0)
    assert abs(s.lower_bound() - lb_ref) <= LB_RTOL * max(abs(lb_ref), float(raw.max()))
    err = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert err < 1e-3, err
    s.close()


@pytest.mark.parametrize("which,chunk,iters", [("config1", 8, 200), ("config2", 16, 300)])
def test_uncapped_splitting_matches_oracle(torch, which, chunk, iters):
    inst = getattr(I, which)()
    prob, d, allowed, fixed, const, dec = _problem(inst, chunk, 0)
    assert B.decompose(prob, fixed, const, chunk, 8).nb < dec.nb  # the default cap would bind
    s = _solver(inst, d, None if inst.topk is None else allowed, split_chunk=chunk, split_max_segments=0)
    assert s.info()["nbdds"] == dec.nb
    s.dual(iters)
    o = S.DualOracle(dec)
    o.iterate(iters)
    lb, ref = s.lower_bound(), o.lower_bound()
    assert abs(lb - ref) <= LB_RTOL * max(abs(ref), 1e-3), (lb, ref)
    np.testing.assert_allclose(s.min_marginals(), o.min_marginals(), atol=MM_ATOL, rtol=0)
    s.close()
