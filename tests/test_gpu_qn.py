"""Quasi-Newton powered MMA (Alg. 1 with Alg. 4-6, ``disco_dual_qn``) against the FP64
oracle (``oracle/lbfgs.py``): the bound after every call matches to 1e-5 relative, with an
absolute floor of 1e-7 (FP32 device arithmetic; the step search compares bounds, so the two
sides take the same decisions except at near-ties, where the bound is flat anyway), never
decreases, and the dual stays feasible (Eq. D)."""
import numpy as np
import pytest

from oracle import bdd as B
from oracle import lbfgs as Q
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


def _setup(which, chunk):
    inst = getattr(I, which)()
    prob, d, allowed = P.make_problem(inst)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, chunk)
    return inst, prob, d, allowed, fixed, dec


def _solver(inst, d, allowed, **kw):
    from paper_2310_08230_gb300.api import Solver

    return Solver(inst.X.T, inst.Y.T, np.asarray(d, np.float32), None if inst.topk is None else allowed, **kw)


@pytest.mark.parametrize("which,chunk,mma", [("tet", 0, 2), ("config1", 0, 3), ("config1", 4, 3), ("config2", 16, 2)])
def test_qn_bounds_match_oracle(torch, which, chunk, mma):
    inst, prob, d, allowed, fixed, dec = _setup(which, chunk)
    qn = Q.QuasiNewton(S.DualOracle(dec), mma_iters=mma)
    s = _solver(inst, d, allowed, split_chunk=chunk, qn_memory=5)
    prev = s.lower_bound()
    for _ in range(5):
        qn.step()
        s.dual_qn(1, mma)
        ref = qn.o.lower_bound()
        lb = s.lower_bound()
        # FP32 rounding of a sum of O(10^3) BDD minima of order 0.1-1 (costs in [0, 1]): the
        # absolute floor 1e-7 matters only while the bound itself is still tiny (early calls)
        assert abs(lb - ref) <= 1e-5 * max(abs(ref), 1e-2), (lb, ref, qn.last)
        # both bounds lie within the parity tolerance of the oracle's non-decreasing sequence
        assert lb >= prev - 2e-5 * max(abs(prev), 1e-2)
        prev = lb
    # Eq. D feasibility: sum_j lambda^j_i + |J_i| pend_i = c_i
    lam, pend = s.get_state()
    free = np.nonzero(fixed < 0)[0]
    tot = np.bincount(dec.layer_var, weights=lam.astype(np.float64), minlength=dec.nvars_total)
    resid = tot[free] + dec.deg[free] * pend[: len(free)].astype(np.float64) - prob.cost[free]
    assert np.abs(resid).max() < 1e-5
    s.close()


def test_converge_with_qn_reaches_the_mma_bound(torch):
    inst, prob, d, allowed, fixed, dec = _setup("config2", 16)
    a = _solver(inst, d, allowed, split_chunk=16)
    b = _solver(inst, d, allowed, split_chunk=16, qn_memory=5)
    na, lba, oka = a.converge(2000)
    nb, lbb, okb = b.converge(2000)
    assert oka and okb
    assert abs(lba - lbb) <= 1e-5 * abs(lba)
    a.close()
    b.close()
