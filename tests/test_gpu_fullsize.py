"""The bench workload itself (5120-triangle icosphere pair, top-16, chunk 32; 6.0 M BDD
nodes), in the launch configuration bench.py times, checked by properties that hold at
any size: the bound never decreases over blocks of iterations, it is bit-identical whether
the pair is solved alone or inside a batch (to 1e-12), quasi-Newton steps reach the same bound, the
rounded matching is feasible (the library checks A x = b exactly) and costs at least the
bound, and the dual state stays finite."""
import numpy as np
import pytest

from synth import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08230_gb300.build import build

    build()
    from paper_2310_08230_gb300.api import candidates, pair_costs

    inst = I.config3()
    d = pair_costs(torch.from_numpy(inst.FX).cuda(), torch.from_numpy(inst.FY).cuda())
    al = candidates(d, inst.topk, inst.X.T, inst.Y.T)
    return inst, d, al


def test_fullsize_properties(setup):
    from paper_2310_08230_gb300.api import Solver

    inst, d, al = setup
    s = Solver(inst.X.T, inst.Y.T, d, al, split_chunk=32)
    info = s.info()
    assert info["nnodes"] > 5_000_000
    prev = s.lower_bound()
    for _ in range(4):
        s.dual(10)
        lb = s.lower_bound()
        assert lb >= prev - 2e-5 * abs(lb)  # two values, each within 1e-5 of a monotone FP64 sequence
        prev = lb
    # alone vs inside a batch with a second pair: same per-lane arithmetic, same bound
    other = I.config2()
    import torch

    from paper_2310_08230_gb300.api import candidates, pair_costs

    d2 = pair_costs(torch.from_numpy(other.FX).cuda(), torch.from_numpy(other.FY).cuda())
    a2 = candidates(d2, other.topk, other.X.T, other.Y.T)
    b = Solver.batch([(inst.X.T, inst.Y.T, d, al), (other.X.T, other.Y.T, d2, a2)], split_chunk=32)
    b.dual(40)
    assert b.lower_bounds()[0] == pytest.approx(s.lower_bound(), rel=1e-12)
    b.close()
    x, cost, ok = s.primal()
    assert ok and cost >= s.lower_bound() - 1e-5 * abs(cost)  # the bound's tolerance
    s.close()


def test_fullsize_qn_reaches_the_bound(setup):
    from paper_2310_08230_gb300.api import Solver

    inst, d, al = setup
    a = Solver(inst.X.T, inst.Y.T, d, al, split_chunk=32)
    q = Solver(inst.X.T, inst.Y.T, d, al, split_chunk=32, qn_memory=5)
    na, lba, oka = a.converge(2000)
    nq, lbq, okq = q.converge(2000)
    assert oka and okq
    assert lbq >= lba - 2e-5 * abs(lba)  # two bounds, each within 1e-5 of its FP64 value
    lam, pend = q.get_state()
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(pend))
    a.close()
    q.close()
