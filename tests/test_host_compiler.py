"""CPU checks of the C ABI library without a GPU: it loads, exports every symbol that
include/disco.h declares, and its host compiler (disco_compile_host) builds the same
problem, presolve and BDD segments as the independently written oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import bdd as B
from oracle import problem as P
from synth import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2310_08230_gb300 import _lib
    from paper_2310_08230_gb300.build import build

    build()
    return _lib


def test_library_exports_every_declared_symbol(L):
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(disco_[a-z_0-9]+)\s*\(", src, re.M))
    assert len(names) >= 15
    lib = L.lib()
    for n in sorted(names):
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, n


def test_struct_layouts_match_header(L):
    assert ctypes.sizeof(L.disco_opts) == 96
    assert ctypes.sizeof(L.disco_info_t) == 160
    assert ctypes.sizeof(L.disco_mesh) == 24


def test_default_options(L):
    o = L.disco_opts()
    assert L.lib().disco_default_opts(ctypes.byref(o)) == 0
    assert o.omega == 0.5 and o.lb_every == 20 and o.split_max_segments == 8
    assert o.graph_iters == 10 and o.autotune == 1 and o.normalize_costs == 1 and o.qn_memory == 0
    assert o.cost_model == 0 and o.tile_order == 0


def _compile(L, inst, allowed, d, chunk, maxseg=8):
    mx = L.disco_mesh(inst.X.nv, inst.X.nt, None, inst.X.T.ctypes.data)
    my = L.disco_mesh(inst.Y.nv, inst.Y.nt, None, inst.Y.T.ctypes.data)
    info = L.disco_info_t()
    d32 = np.ascontiguousarray(d, np.float32)
    a8 = None if allowed is None else np.ascontiguousarray(allowed, np.uint8)
    args = (ctypes.byref(mx), ctypes.byref(my), d32.ctypes.data, None if a8 is None else a8.ctypes.data, chunk, maxseg,
            ctypes.byref(info))
    L.check(L.lib().disco_compile_host(*args, None, None, 0, None, 0), "compile")
    sv = np.empty(info.nslots, np.int32)
    sw = np.empty(info.nslots, np.int32)
    fx = np.empty(info.nvars, np.int8)
    L.check(L.lib().disco_compile_host(*args, sv.ctypes.data, sw.ctypes.data, sv.shape[0], fx.ctypes.data,
                                       fx.shape[0]), "compile")
    return info, sv, sw, fx


@pytest.mark.parametrize("which,chunk,maxseg", [("tet", 0, 8), ("tet", 5, 8), ("tet", 5, 0), ("config1", 0, 8),
                                                ("config1", 7, 8), ("config1", 7, 3), ("config2", 0, 8),
                                                ("config2", 16, 8), ("config2", 16, 0)])
def test_host_compiler_matches_oracle(L, which, chunk, maxseg):
    inst = getattr(I, which)()
    prob, d, allowed = P.make_problem(inst)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, chunk, maxseg)
    info, sv, sw, fx = _compile(L, inst, None if inst.topk is None else allowed, d, chunk, maxseg)
    assert info.nvars == prob.nvars
    assert info.nrows == prob.nrows
    assert np.array_equal(fx, fixed)
    assert info.nvars_free == int((fixed < 0).sum())
    assert info.nvars_aux == dec.nvars_total - dec.nvars
    assert info.nbdds == dec.nb
    assert np.array_equal(sv, dec.layer_var)
    assert np.array_equal(sw, np.diff(dec.layer_node_ptr))
    assert info.nnodes == dec.n_nodes
    assert info.constant == pytest.approx(const, abs=1e-6)


def test_host_compiler_errors(L):
    inst = I.config1()
    d = np.ones((inst.X.nv, inst.Y.nv), np.float32)
    info = L.disco_info_t()
    mx = L.disco_mesh(inst.X.nv, inst.X.nt, None, inst.X.T.ctypes.data)
    # genus mismatch: torus vs icosahedron
    from synth import meshes as M
    t = M.torus(3, 4)
    mt = L.disco_mesh(t.nv, t.nt, None, t.T.ctypes.data)
    dt = np.ones((inst.X.nv, t.nv), np.float32)
    rc = L.lib().disco_compile_host(ctypes.byref(mx), ctypes.byref(mt), dt.ctypes.data, None, 0, 8,
                                    ctypes.byref(info), None, None, 0, None, 0)
    assert rc == L.DISCO_ERR_GENUS_MISMATCH
    # flipped triangle
    T = inst.Y.T.copy()
    T[0] = T[0][[0, 2, 1]]
    my = L.disco_mesh(inst.Y.nv, inst.Y.nt, None, T.ctypes.data)
    rc = L.lib().disco_compile_host(ctypes.byref(mx), ctypes.byref(my), d.ctypes.data, None, 0, 8,
                                    ctypes.byref(info), None, None, 0, None, 0)
    assert rc == L.DISCO_ERR_NONMANIFOLD
    # negative / NaN costs
    bad = d.copy()
    bad[0, 0] = np.nan
    my = L.disco_mesh(inst.Y.nv, inst.Y.nt, None, inst.Y.T.ctypes.data)
    rc = L.lib().disco_compile_host(ctypes.byref(mx), ctypes.byref(my), bad.ctypes.data, None, 0, 8,
                                    ctypes.byref(info), None, None, 0, None, 0)
    assert rc == L.DISCO_ERR_INVALID_ARG
    # a candidate mask that leaves a triangle without any element
    allowed = np.zeros((inst.X.nv, inst.Y.nv), np.uint8)
    rc = L.lib().disco_compile_host(ctypes.byref(mx), ctypes.byref(my), d.ctypes.data, allowed.ctypes.data, 0, 8,
                                    ctypes.byref(info), None, None, 0, None, 0)
    assert rc == L.DISCO_ERR_INFEASIBLE
    assert b"element" in L.lib().disco_last_error() or b"empty" in L.lib().disco_last_error()


@pytest.mark.slow
def test_host_compiler_matches_oracle_at_full_size(L):
    """The benchmark workload (5120-triangle icosphere pair, top-16, chunk 32, the default cap
    of 8 segments per row): product space, presolve fixings, every segment's variables and
    widths, auxiliary variables and node count, bit for bit (about 75 s of oracle time)."""
    inst = I.config3()
    d32 = P.pair_distance(inst.FX, inst.FY).astype(np.float32)
    allowed = P.candidate_pairs(d32.astype(np.float64), inst.topk, inst.X.T, inst.Y.T)
    prob = P.build_problem(inst.X.T, inst.Y.T, d32.astype(np.float64), allowed)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 32, 8)
    info, sv, sw, fx = _compile(L, inst, allowed, d32, 32, 8)
    assert info.nvars == prob.nvars and info.nrows == prob.nrows
    assert np.array_equal(fx, fixed)
    assert info.nvars_free == int((fixed < 0).sum())
    assert info.nvars_aux == dec.nvars_total - dec.nvars
    assert info.nbdds == dec.nb
    assert np.array_equal(sv, dec.layer_var)
    assert np.array_equal(sw, np.diff(dec.layer_node_ptr))
    assert info.nnodes == dec.n_nodes == 6019316
    assert info.constant == pytest.approx(const, abs=1e-6)


_POISON_SCRIPT = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2310_08230_gb300 import _lib as L
from oracle import problem as P
from synth import instances as I
inst = I.config3()
d32 = P.pair_distance(inst.FX, inst.FY).astype(np.float32)
a8 = P.candidate_pairs(d32.astype(np.float64), inst.topk, inst.X.T, inst.Y.T).astype(np.uint8)
mx = L.disco_mesh(inst.X.nv, inst.X.nt, None, inst.X.T.ctypes.data)
my = L.disco_mesh(inst.Y.nv, inst.Y.nt, None, inst.Y.T.ctypes.data)
info = L.disco_info_t()
args = (ctypes.byref(mx), ctypes.byref(my), d32.ctypes.data, a8.ctypes.data, 32, 8, ctypes.byref(info))
L.check(L.lib().disco_compile_host(*args, None, None, 0, None, 0), "compile")
sv = np.empty(info.nslots, np.int32); sw = np.empty(info.nslots, np.int32); fx = np.empty(info.nvars, np.int8)
L.check(L.lib().disco_compile_host(*args, sv.ctypes.data, sw.ctypes.data, sv.shape[0], fx.ctypes.data, fx.shape[0]), "compile")
np.savez(sys.argv[2], sv=sv, sw=sw, fx=fx, meta=np.array([info.nvars, info.nrows, info.nvars_free, info.nvars_aux,
         info.nbdds, info.nnodes], np.int64), constant=np.array([info.constant]))
"""


@pytest.mark.slow
def test_host_compiler_ignores_block_contents(L, tmp_path):
    """Large host blocks are reused across builds without being cleared, so no step of the
    compiler may depend on what a block held before: with every block filled with 0xA5 when
    handed out (DISCO_HOST_CACHE_POISON), the 5120-triangle plan is the same bit for bit."""
    import subprocess
    import sys

    inst = I.config3()
    d32 = P.pair_distance(inst.FX, inst.FY).astype(np.float32)
    allowed = P.candidate_pairs(d32.astype(np.float64), inst.topk, inst.X.T, inst.Y.T)
    info, sv, sw, fx = _compile(L, inst, allowed, d32, 32, 8)
    out = str(tmp_path / "poisoned.npz")
    env = dict(os.environ, DISCO_HOST_CACHE_POISON="1")
    subprocess.run([sys.executable, "-c", _POISON_SCRIPT, ROOT, out], env=env, cwd=ROOT, check=True, timeout=600)
    z = np.load(out)
    assert list(z["meta"]) == [info.nvars, info.nrows, info.nvars_free, info.nvars_aux, info.nbdds, info.nnodes]
    assert z["constant"][0] == info.constant
    assert np.array_equal(z["sv"], sv) and np.array_equal(z["sw"], sw) and np.array_equal(z["fx"], fx)


def _batch_pair(k):
    return I.config4(64)[k]


@pytest.mark.parametrize("which", ["config1-top4", "config2", "batch5", "batch17", "truth-only", "bipyramid12-random",
                                   "bipyramid16-random", "config2-random"])
def test_dense_and_sparse_enumeration_give_the_same_plan(L, monkeypatch, which):
    """The product space is enumerated either from the candidate rows (a bit lookup per
    candidate corner pair) or by AND-ing per-vertex bit sets over Y triangles and edges; the
    compiler picks one by an operation count. Both must give the same elements in the same
    canonical order: the plan (fixings per element, every segment's variables and widths,
    constant) is compared bit for bit with each path forced (DISCO_HOST_ENUM)."""
    if which == "config1-top4":
        inst = I.config1()
        k = 4
    elif which.startswith("batch"):
        inst = _batch_pair(int(which[5:]))
        k = inst.topk
    else:
        inst = I.config2()
        k = inst.topk
    if which.startswith("bipyramid"):
        inst = I.bipyramid_pair(int(which[9:11]))  # apexes of valence 12 / 16
    d32 = P.pair_distance(inst.FX, inst.FY).astype(np.float32)
    if which == "truth-only":
        allowed = np.zeros((inst.X.nv, inst.Y.nv), bool)
        allowed[np.arange(inst.X.nv), inst.perm] = True
    elif which.endswith("-random"):
        # irregular masks: each pair kept with probability 0.6 (bipyramids) or 0.3, plus the
        # ground truth so that every triangle keeps an element
        rng = np.random.Generator(np.random.PCG64(len(which)))
        allowed = rng.random((inst.X.nv, inst.Y.nv)) < (0.6 if which.startswith("bipyramid") else 0.3)
        allowed[np.arange(inst.X.nv), inst.perm] = True
    else:
        allowed = P.candidate_pairs(d32.astype(np.float64), k, inst.X.T, inst.Y.T)
    plans = {}
    for mode in ("sparse", "dense"):
        monkeypatch.setenv("DISCO_HOST_ENUM", mode)
        plans[mode] = _compile(L, inst, allowed, d32, 32, 8)
    (ia, sva, swa, fxa), (ib, svb, swb, fxb) = plans["sparse"], plans["dense"]
    assert (ia.nvars, ia.nrows, ia.nvars_free, ia.nvars_aux, ia.nbdds, ia.nnodes) == \
        (ib.nvars, ib.nrows, ib.nvars_free, ib.nvars_aux, ib.nbdds, ib.nnodes)
    assert ia.constant == ib.constant
    assert np.array_equal(fxa, fxb) and np.array_equal(sva, svb) and np.array_equal(swa, swb)


@pytest.mark.parametrize("which", ["tet", "config1", "config2"])
def test_host_compiler_when_presolve_fixes_everything(L, which):
    """With only the ground-truth vertex pairs allowed, the product space is the true
    triangle pairs (a degenerate element needs two X corners on one Y vertex), every
    projection row holds one element, and presolve fixes all of them to 1: no free variable,
    no BDD, a constant equal to the sum of the normalised costs (Sec. 3.1, Eq. P)."""
    inst = getattr(I, which)()
    d32 = P.pair_distance(inst.FX, inst.FY).astype(np.float32)
    allowed = np.zeros((inst.X.nv, inst.Y.nv), bool)
    allowed[np.arange(inst.X.nv), inst.perm] = True
    prob = P.build_problem(inst.X.T, inst.Y.T, d32.astype(np.float64), allowed)
    fixed, const = P.presolve(prob)
    assert prob.nvars == inst.X.nt and np.all(fixed == 1)
    info, sv, sw, fx = _compile(L, inst, allowed, d32, 0, 8)
    assert info.nvars == prob.nvars and info.nvars_free == 0 and info.nbdds == 0 and info.nslots == 0
    assert np.array_equal(fx, fixed)
    assert info.constant == pytest.approx(prob.cost.sum(), rel=1e-12)
