"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (FP32 device arithmetic on costs normalised to [0, 1]): lower bound 1e-5
relative after a fixed iteration count, min-marginals 1e-4 absolute, primal feasible
exactly with cost within 1e-4 relative of the oracle's (ties excepted), pair costs 1e-5
relative."""
import numpy as np
import pytest

from oracle import bdd as B
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


_cache = {}


def _oracle(which, chunk):
    key = (which, chunk)
    if key not in _cache:
        inst = getattr(I, which)()
        prob, d, allowed = P.make_problem(inst)
        fixed, const = P.presolve(prob)
        dec = B.decompose(prob, fixed, const, chunk)
        _cache[key] = (inst, prob, d, allowed, fixed, dec)
    return _cache[key]


def _solver(inst, d, allowed, **kw):
    from paper_2310_08230_gb300.api import Solver

    return Solver(inst.X.T, inst.Y.T, np.asarray(d, np.float32), None if inst.topk is None else allowed, **kw)


def test_pair_costs_match_oracle(torch):
    from paper_2310_08230_gb300.api import pair_costs

    for which in ("config1", "config2"):
        inst = getattr(I, which)()
        d_ref = P.pair_distance(inst.FX, inst.FY)
        d = pair_costs(torch.from_numpy(inst.FX).cuda(), torch.from_numpy(inst.FY).cuda())
        torch.cuda.synchronize()
        np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-5, atol=1e-7)


def test_pair_costs_ragged_tiles(torch):
    """Sizes that are not multiples of the 64 x 64 tile or the 32-wide k chunk."""
    from paper_2310_08230_gb300.api import pair_costs

    rng = np.random.Generator(np.random.PCG64(7))
    for nx, ny, D in ((1, 1, 1), (65, 3, 33), (130, 97, 70)):
        FX = rng.standard_normal((nx, D)).astype(np.float32)
        FY = rng.standard_normal((ny, D)).astype(np.float32)
        d = pair_costs(torch.from_numpy(FX).cuda(), torch.from_numpy(FY).cuda()).cpu().numpy()
        np.testing.assert_allclose(d, P.pair_distance(FX, FY), rtol=1e-5, atol=1e-7)


def test_pair_costs_from_host_arrays(torch):
    """disco_pair_costs and disco_pair_distances take host feature arrays (copied in by the
    library) as well as device ones, with the same results."""
    from paper_2310_08230_gb300 import _lib as L

    inst = I.config2()
    FX = np.ascontiguousarray(inst.FX)
    FY = np.ascontiguousarray(inst.FY)
    nvx, nvy, D = FX.shape[0], FY.shape[0], FX.shape[1]
    lib = L.lib()
    for fn, ref in ((lib.disco_pair_costs, P.pair_distance(FX, FY)),
                    (lib.disco_pair_distances, P.pair_euclid(FX, FY))):
        got = []
        for fx, fy in ((FX, FY), (torch.from_numpy(FX).cuda(), FY), (torch.from_numpy(FX).cuda(),
                                                                     torch.from_numpy(FY).cuda())):
            d = torch.empty((nvx, nvy), dtype=torch.float32, device="cuda")
            px = fx.ctypes.data if isinstance(fx, np.ndarray) else fx.data_ptr()
            py = fy.ctypes.data if isinstance(fy, np.ndarray) else fy.data_ptr()
            L.check(fn(px, py, nvx, nvy, D, d.data_ptr(), None), "pair kernel")
            torch.cuda.synchronize()
            got.append(d.cpu().numpy())
        np.testing.assert_array_equal(got[0], got[2])
        np.testing.assert_array_equal(got[1], got[2])
        np.testing.assert_allclose(got[2], ref, rtol=1e-5, atol=1e-7)


def test_candidates_match_oracle(torch):
    from paper_2310_08230_gb300.api import candidates

    for which in ("config2",):
        inst = getattr(I, which)()
        d_ref = P.pair_distance(inst.FX, inst.FY)
        # both sides rank the same FP32 distances: take the decision in one precision
        d32 = d_ref.astype(np.float32)
        ref = P.candidate_pairs(d32.astype(np.float64), inst.topk, inst.X.T, inst.Y.T)
        got = candidates(torch.from_numpy(d32).cuda(), inst.topk, inst.X.T, inst.Y.T).cpu().numpy().astype(bool)
        assert np.array_equal(got, ref)
        assert np.all(got[np.arange(inst.X.nv), inst.perm])


@pytest.mark.parametrize("which,chunk,iters", [("tet", 0, 0), ("tet", 0, 50), ("tet", 5, 50), ("config1", 0, 0),
                                               ("config1", 0, 200), ("config1", 8, 200), ("config2", 0, 0),
                                               ("config2", 0, 500)])
def test_lower_bound_parity(torch, which, chunk, iters):
    inst, prob, d, allowed, fixed, dec = _oracle(which, chunk)
    o = S.DualOracle(dec)
    o.iterate(iters)
    s = _solver(inst, d, allowed, split_chunk=chunk)
    s.dual(iters)
    lb = s.lower_bound()
    ref = o.lower_bound()
    assert abs(lb - ref) <= LB_RTOL * max(abs(ref), 1e-3), (lb, ref)
    info = s.info()
    assert info["nslots"] == dec.n_layers and info["nnodes"] == dec.n_nodes
    s.close()


@pytest.mark.parametrize("which,chunk,iters", [("tet", 0, 30), ("config1", 0, 100), ("config1", 8, 60),
                                               ("config2", 0, 100)])
def test_min_marginal_parity(torch, which, chunk, iters):
    inst, prob, d, allowed, fixed, dec = _oracle(which, chunk)
    o = S.DualOracle(dec)
    o.iterate(iters)
    s = _solver(inst, d, allowed, split_chunk=chunk)
    s.dual(iters)
    mm = s.min_marginals()
    ref = o.min_marginals()
    np.testing.assert_allclose(mm, ref, atol=MM_ATOL, rtol=0)
    s.close()


def test_state_roundtrip_and_dual_feasibility(torch):
    inst, prob, d, allowed, fixed, dec = _oracle("config1", 0)
    s = _solver(inst, d, allowed)
    s.dual(37)
    lam, pend = s.get_state()
    # sum_j lambda^j_i + |J_i| pend_i = c_i (Eq. D feasibility), in FP32
    free = np.nonzero(fixed < 0)[0]
    lv = dec.layer_var
    tot = np.bincount(lv, weights=lam.astype(np.float64), minlength=dec.nvars_total)
    resid = tot[free] + dec.deg[free] * pend[: len(free)].astype(np.float64) - prob.cost[free]
    assert np.abs(resid).max() < 1e-5
    lb1 = s.lower_bound()
    s2 = _solver(inst, d, allowed)
    s2.set_state(lam, pend)
    assert s2.lower_bound() == pytest.approx(lb1, rel=1e-6)
    s.dual(5)
    s2.dual(5)
    assert s2.lower_bound() == pytest.approx(s.lower_bound(), rel=1e-6)
    s.close()
    s2.close()


@pytest.mark.parametrize("which,chunk", [("config1", 0), ("config2", 16)])
def test_graph_replay_and_launch_geometries_are_bit_identical(torch, which, chunk):
    """Plain launches with the default geometry, graph replay, and the autotuner (which runs
    its trial iterations in every geometry) give bit-identical dual states."""
    from paper_2310_08230_gb300 import _lib as L

    inst, prob, d, allowed, fixed, dec = _oracle(which, chunk)
    states = []
    for kw in (dict(graph_iters=0, autotune=0), dict(graph_iters=10, autotune=0), dict(graph_iters=7, autotune=1)):
        s = _solver(inst, d, allowed, split_chunk=chunk, **kw)
        n0 = L.lib().disco_kernel_launches()
        s.dual(6)   # autotune trials when enabled
        s.dual(33)  # graph blocks plus a plain remainder
        launched = L.lib().disco_kernel_launches() - n0
        info = s.info()
        assert info["iterations"] == 39
        assert info["launch_geometry"] in (1, 2, 4)
        assert launched >= 2 * 39  # every replayed kernel is counted
        lam, pend = s.get_state()
        states.append((lam, pend, s.lower_bound(), s.min_marginals()))
        s.close()
    for lam, pend, lb, mm in states[1:]:
        np.testing.assert_array_equal(lam, states[0][0])
        np.testing.assert_array_equal(pend, states[0][1])
        assert lb == states[0][2]
        np.testing.assert_array_equal(mm, states[0][3])


def test_bound_is_monotone_and_below_primal(torch):
    inst, prob, d, allowed, fixed, dec = _oracle("config2", 0)
    s = _solver(inst, d, allowed)
    prev = s.lower_bound()
    for _ in range(10):
        s.dual(10)
        lb = s.lower_bound()
        assert lb >= prev - 2e-5 * abs(lb)  # two values, each within LB_RTOL of a monotone FP64 sequence
        prev = lb
    x, cost, ok = s.primal()
    assert ok
    assert not np.any(prob.residual(x))
    assert prev <= cost + LB_RTOL * abs(cost)  # FP64 bound <= OPT <= cost; the GPU bound is within LB_RTOL
    s.close()


@pytest.mark.parametrize("which,iters", [("tet", 50), ("config1", 200), ("config2", 500)])
def test_primal_parity(torch, which, iters):
    inst, prob, d, allowed, fixed, dec = _oracle(which, 0)
    o = S.DualOracle(dec)
    o.iterate(iters)
    ref = PR.round_primal(o, prob, fixed)
    s = _solver(inst, d, allowed)
    s.dual(iters)
    x, cost, ok = s.primal()
    assert ok and ref.ok
    assert not np.any(prob.residual(x))  # integer-exact feasibility
    # the library's c comes from FP32 pair costs; the oracle's from FP64 features
    assert cost == pytest.approx(float(prob.cost @ x), rel=1e-6)
    assert abs(cost - ref.cost) <= 1e-4 * abs(ref.cost)
    s.close()


def test_converge_stops_on_relative_change(torch):
    inst, prob, d, allowed, fixed, dec = _oracle("config2", 0)
    s = _solver(inst, d, allowed, lb_every=20, conv_rel_tol=1e-6)
    n, lb, ok = s.converge(5000)
    assert ok and n % 20 == 0 and n > 0
    s.dual(20)
    assert abs(s.lower_bound() - lb) < 1e-5 * abs(lb)
    s.close()


def test_errors_are_codes_not_crashes(torch):
    from paper_2310_08230_gb300 import _lib as L

    inst, prob, d, allowed, fixed, dec = _oracle("tet", 0)
    s = _solver(inst, d, allowed)
    small = np.zeros(3, np.float32)
    rc = L.lib().disco_min_marginals(s.h, small.ctypes.data, 3)
    assert rc == L.DISCO_ERR_INVALID_ARG
    rc = L.lib().disco_dual(s.h, -1)
    assert rc == L.DISCO_ERR_INVALID_ARG
    s.dual(3)
    assert np.isfinite(s.lower_bound())
    s.close()


@pytest.mark.parametrize("scale", [1e6, 1e13])
def test_unnormalised_costs_of_any_scale(torch, scale):
    """The averaging grid follows the largest cost (2^-F with 2^(32 - F) above it), so raw
    costs far from [0, 1] still match the oracle to the bound tolerance."""
    inst, prob, d, allowed, fixed, dec = _oracle("config1", 0)
    d2 = (d * scale).astype(np.float32)
    p2 = P.build_problem(inst.X.T, inst.Y.T, d2.astype(np.float64), None, normalize=False)
    f2, c2 = P.presolve(p2)
    o = S.DualOracle(B.decompose(p2, f2, c2, 0))
    o.iterate(60)
    s = _solver(inst, d2, allowed, normalize_costs=0)
    s.dual(60)
    lb, ref = s.lower_bound(), o.lower_bound()
    assert abs(lb - ref) <= LB_RTOL * abs(ref), (lb, ref)
    s.close()


def test_out_of_range_state_is_reported(torch):
    """A deferred mean outside the averaging sums' range (here imported by set_state) is
    clamped and flagged: the next synchronising call raises DISCO_ERR_RANGE, and the handle
    works again once a valid state is set."""
    from paper_2310_08230_gb300 import _lib as L

    inst, prob, d, allowed, fixed, dec = _oracle("tet", 0)
    s = _solver(inst, d, allowed)
    s.dual(10)
    lam, pend = s.get_state()
    lb = s.lower_bound()
    bad = pend.copy()
    bad[0] = 1e30
    s.set_state(lam, bad)
    with pytest.raises(L.DiscoError) as e:
        s.lower_bound()
    assert e.value.code == L.DISCO_ERR_RANGE
    s.set_state(lam, pend)
    assert s.lower_bound() == pytest.approx(lb, rel=1e-6)
    s.close()


@pytest.mark.parametrize("which", ["tet", "config1", "config2"])
def test_instance_that_presolve_solves(torch, which):
    """Only the ground-truth pairs allowed: presolve fixes every element (no slot, no tile).
    The bound is the constant at any iteration count, rounding returns the true matching,
    and d(bound)/d(pair costs) is the closed form of the bound sum_e c_e / c_max over the
    fixed elements, c_e the mean of e's three pair costs (Sec. 3.1; Eq. D with no BDD)."""
    inst = getattr(I, which)()
    d32 = P.pair_distance(inst.FX, inst.FY).astype(np.float32)
    d = d32.astype(np.float64)
    allowed = np.zeros((inst.X.nv, inst.Y.nv), bool)
    allowed[np.arange(inst.X.nv), inst.perm] = True
    prob = P.build_problem(inst.X.T, inst.Y.T, d, allowed)
    raw = sum(d[prob.vm[:, v], prob.vn[:, v]] for v in range(3)) / 3.0
    C, cmax, emax = raw.sum(), raw.max(), int(np.argmax(raw))
    from paper_2310_08230_gb300.api import Solver

    s = Solver(inst.X.T, inst.Y.T, d32, allowed.astype(np.uint8))
    assert s.info()["nslots"] == 0 and s.info()["nvars_free"] == 0
    for iters in (0, 5):
        s.dual(iters)
        assert s.lower_bound() == pytest.approx(C / cmax, rel=1e-12)
    assert s.min_marginals().shape == (0,)
    x, cost, ok = s.primal()
    assert ok and np.all(x == 1) and not np.any(prob.residual(x))
    assert cost == pytest.approx(C / cmax, rel=1e-12)
    s.record(10, 5)
    g = s.grad().reshape(inst.X.nv, inst.Y.nv).astype(np.float64)
    ref = np.zeros_like(g)
    for v in range(3):
        np.add.at(ref, (prob.vm[:, v], prob.vn[:, v]), 1.0 / (3.0 * cmax))
        ref[prob.vm[emax, v], prob.vn[emax, v]] -= C / (3.0 * cmax * cmax)
    assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max()
    s.close()
