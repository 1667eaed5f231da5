"""Pins of the oracle's candidate rules (Sec. 4: the product space pruned to neighbourhoods
of vertex matches) and of its point map, each against values derived by hand or from the
mesh geometry, never from the oracle's own ring helper; and planted mistakes (no dilation,
dilation on the wrong mesh, one direction dropped, rings off by one, the coarse-to-fine map
forgotten, pairs not deduplicated) that each pin must catch."""
import numpy as np
import pytest

from oracle import problem as P
from synth import instances as I
from synth import meshes as M

# The octahedron, typed out: 0 = +x, 1 = -x, 2 = +y, 3 = -y, 4 = +z, 5 = -z, faces
# counter-clockwise seen from outside. Each vertex is adjacent to every other except its
# antipode, so its closed 1-ring is everything but the antipode.
OCTA_T = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                   [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], np.int32)
ANTIPODE = [1, 0, 3, 2, 5, 4]
OCTA_RING1 = np.array([[v != ANTIPODE[u] for v in range(6)] for u in range(6)])


def _geometric_ring(mesh: M.Mesh) -> np.ndarray:
    """Closed 1-ring of a mesh whose edges all have the shortest vertex distance (the
    icosahedron): two vertices are adjacent iff their distance is that length."""
    V = mesh.V.astype(np.float64)
    D = np.linalg.norm(V[:, None, :] - V[None, :, :], axis=2)
    e = D[D > 0].min()
    return D < 1.001 * e


def _exact_copy():
    """The icosahedron against a relabelled copy whose features are X's permuted, with no
    noise: d(m, perm[m]) = 0 and every other cost is positive."""
    rng = np.random.Generator(np.random.PCG64(3))
    X = M.icosahedron()
    Y, perm = M.relabel(X, rng)
    FX = rng.standard_normal((X.nv, 16))
    FY = np.empty_like(FX)
    FY[perm] = FX
    d = ((FX[:, None, :] - FY[None, :, :]) ** 2).mean(-1)
    return X, Y, perm, d


# ---------------------------------------------------------------------------------------
# planted mistakes, in the oracle, on the CPU


def _plant_no_dilation(mp):
    mp.setattr(P, "closed_one_ring", lambda nv, T: np.eye(nv, dtype=bool))


def _plant_wrong_mesh(mp, TX, TY):
    orig = P.closed_one_ring
    other = {id(TX): TY, id(TY): TX}
    mp.setattr(P, "closed_one_ring", lambda nv, T: orig(nv, other[id(T)]))


def _plant_drop(mp, which):
    orig = P.nearest_indicators

    def f(d, k):
        cxy, cyx = orig(d, k)
        return (np.zeros_like(cxy), cyx) if which == "xy" else (cxy, np.zeros_like(cyx))

    mp.setattr(P, "nearest_indicators", f)


# ---------------------------------------------------------------------------------------
# candidate_pairs


def _tet_pin(k):
    X = M.tetrahedron()
    d = np.random.default_rng(k).random((4, 4))
    return bool(P.candidate_pairs(d, k, X.T, X.T).all())


@pytest.mark.parametrize("k", [1, 2, 4])
def test_tetrahedron_allows_every_pair(k):
    """Every closed 1-ring of the tetrahedron is the whole mesh, so any pick allows all."""
    assert _tet_pin(k)


def _copy_pin():
    X, Y, perm, d = _exact_copy()
    inv = np.argsort(perm)
    ring = _geometric_ring(X)
    # the pick of row m is perm[m] and of column n is inv[n]: (m, n) is allowed iff inv[n]
    # lies in m's closed 1-ring (either direction gives that set)
    want = ring[:, inv]
    return np.array_equal(P.candidate_pairs(d, 1, X.T, Y.T), want), X, Y


def test_exact_copy_k1_is_the_permuted_ring_adjacency():
    ok, _, _ = _copy_pin()
    assert ok


def _one_direction_case(direction):
    """A cost matrix in which pair (m0, n0) is allowed through one direction only."""
    X, Y, perm, d = _exact_copy()
    inv = np.argsort(perm)
    ringY = _geometric_ring(Y)
    m0, n0 = 0, int(perm[0])
    far = int(np.nonzero(~ringY[n0])[0][0])  # a Y vertex not in n0's closed 1-ring
    d = d + 1.0
    if direction == "yx":
        # column n0's nearest is m0 (as before), but row m0's nearest is `far`
        d[m0, far] = 0.5
    else:
        # row m0's nearest is n0, but column n0's nearest is an X vertex far from m0
        ringX = _geometric_ring(X)
        mfar = int(np.nonzero(~ringX[m0])[0][0])
        d[mfar, n0] = 0.5
    return X, Y, d, m0, n0


@pytest.mark.parametrize("direction", ["yx", "xy"])
def test_pair_admitted_by_one_direction_only(direction):
    X, Y, d, m0, n0 = _one_direction_case(direction)
    assert P.candidate_pairs(d, 1, X.T, Y.T)[m0, n0]


def test_only_finite_costs_are_ranked():
    """A row of infinities picks nothing; its pairs come from the columns' picks only."""
    X, Y, perm, d = _exact_copy()
    inv = np.argsort(perm)
    ring = _geometric_ring(X)
    d = d.copy()
    d[0, :] = np.inf
    got = P.candidate_pairs(d, 1, X.T, Y.T)
    want = ring[:, inv]
    keep = np.ones(d.shape, bool)
    keep[:, perm[0]] = False  # column perm[0] lost its zero; its pick is some other vertex
    assert np.array_equal(got[keep], want[keep])
    # row 0 picks nothing itself: with its own pick perm[0] it would also reach the ring of
    # perm[0] on Y; without it, (0, n) needs inv[n] in 0's ring
    cxy, _ = P.nearest_indicators(d, 1)
    assert cxy[0].sum() == 0 and cxy[1:].sum() == d.shape[0] - 1


def test_candidate_pins_catch_planted_mistakes(monkeypatch):
    with monkeypatch.context() as mp:
        _plant_no_dilation(mp)
        assert not _tet_pin(1)
        assert not _copy_pin()[0]
    X, Y, perm, d = _exact_copy()
    with monkeypatch.context() as mp:
        _plant_wrong_mesh(mp, X.T, Y.T)
        assert not np.array_equal(P.candidate_pairs(d, 1, X.T, Y.T), _geometric_ring(X)[:, np.argsort(perm)])
    for direction, dropped in (("yx", "yx"), ("xy", "xy")):
        Xm, Ym, dd, m0, n0 = _one_direction_case(direction)
        with monkeypatch.context() as mp:
            _plant_drop(mp, dropped)
            assert not P.candidate_pairs(dd, 1, Xm.T, Ym.T)[m0, n0]


# ---------------------------------------------------------------------------------------
# coarse_to_fine_candidates


def _c2f(pairs, cx, cy, rings, TX=OCTA_T, TY=OCTA_T, nx=6, ny=6):
    return P.coarse_to_fine_candidates(np.asarray(pairs), np.asarray(cx), np.asarray(cy), rings, TX, nx, TY, ny)


def _c2f_pins():
    out = []
    # no rings: exactly the mapped coarse pairs (coarse (0,0) -> fine (4,1), (1,2) -> (0,5))
    want0 = np.zeros((6, 6), bool)
    want0[4, 1] = want0[0, 5] = True
    out.append(np.array_equal(_c2f([[0, 0], [1, 2]], [4, 0], [1, 3, 5], 0), want0))
    # one ring: the product of the two within-1 sets, typed from the octahedron's antipodes
    want1 = np.outer(OCTA_RING1[4], OCTA_RING1[5])
    out.append(np.array_equal(_c2f([[0, 1]], [4], [0, 5], 1), want1))
    # two rings cover the octahedron (its diameter is 2)
    out.append(bool(_c2f([[0, 1]], [4], [0, 5], 2).all()))
    return out


def test_coarse_to_fine_hand_built_cases():
    assert all(_c2f_pins())


def test_coarse_to_fine_on_the_icosphere_levels():
    """On the 80 -> 320 triangle icosphere pair: no rings give exactly the mapped ground-truth
    pairs; one ring contains every fine ground-truth pair (a midpoint vertex is one edge from
    both ends of its coarse edge, on either mesh)."""
    coarse, fine, cx, cy = I.coarse_fine_pair(2)
    gt = np.stack([np.arange(coarse.X.nv), coarse.perm], 1)
    m0 = P.coarse_to_fine_candidates(gt, cx, cy, 0, fine.X.T, fine.X.nv, fine.Y.T, fine.Y.nv)
    want = np.zeros((fine.X.nv, fine.Y.nv), bool)
    want[cx[gt[:, 0]], cy[gt[:, 1]]] = True
    assert np.array_equal(m0, want)
    m1 = P.coarse_to_fine_candidates(gt, cx, cy, 1, fine.X.T, fine.X.nv, fine.Y.T, fine.Y.nv)
    assert m1[np.arange(fine.X.nv), fine.perm].all()
    assert m1.mean() < 0.2


def test_coarse_to_fine_pins_catch_planted_mistakes(monkeypatch):
    orig = P.coarse_to_fine_candidates
    # rings off by one
    with monkeypatch.context() as mp:
        mp.setattr(P, "coarse_to_fine_candidates",
                   lambda pairs, cx, cy, rings, *a: orig(pairs, cx, cy, max(rings - 1, 0), *a))
        assert not all(_c2f_pins())
    # the coarse-to-fine map forgotten (coarse ids used as fine ids)
    with monkeypatch.context() as mp:
        mp.setattr(P, "coarse_to_fine_candidates",
                   lambda pairs, cx, cy, rings, *a: orig(pairs, np.arange(6), np.arange(6), rings, *a))
        assert not all(_c2f_pins())
    # the ring taken on one side only: the oracle builds X's relation first, then Y's
    with monkeypatch.context() as mp:
        ring = P.closed_one_ring
        calls = []

        def x_side_only(nv, T):
            calls.append(nv)
            return ring(nv, T) if len(calls) % 2 == 1 else np.eye(nv, dtype=bool)

        mp.setattr(P, "closed_one_ring", x_side_only)
        assert not all(_c2f_pins())


# ---------------------------------------------------------------------------------------
# point_map


class _Elems:
    """Just the corner arrays of a problem: what point_map reads."""

    def __init__(self, vm, vn):
        self.vm = np.asarray(vm)
        self.vn = np.asarray(vn)


def _point_map_pin():
    # e0 tri-tri; e1 shares two corner pairs with e0; e2 repeats a pair inside itself (a
    # degenerate element); e3 is not selected
    prob = _Elems([[0, 1, 2], [2, 3, 0], [4, 4, 1], [5, 5, 5]], [[5, 6, 7], [7, 7, 5], [8, 8, 9], [0, 0, 0]])
    got = P.point_map(prob, np.array([1, 1, 1, 0]))
    want = np.array([[0, 5], [1, 6], [1, 9], [2, 7], [3, 7], [4, 8]])
    return got.shape == want.shape and np.array_equal(got, want)


def test_point_map_hand_built():
    assert _point_map_pin()
    empty = P.point_map(_Elems([[0, 1, 2]], [[3, 4, 5]]), np.array([0]))
    assert empty.shape == (0, 2)


def test_point_map_of_the_ground_truth_matching():
    """The corner pairs of the relabelled identity are exactly the ground-truth vertex map."""
    inst = I.config1()
    prob, _, _ = P.make_problem(inst)
    tt = np.nonzero(prob.vtype == P.TT)[0]
    x = np.zeros(prob.nvars, np.int64)
    x[tt[np.all(inst.perm[prob.vm[tt]] == prob.vn[tt], axis=1)]] = 1
    got = P.point_map(prob, x)
    assert np.array_equal(got, np.stack([np.arange(inst.X.nv), inst.perm], 1))


def test_point_map_pin_catches_planted_mistakes(monkeypatch):
    with monkeypatch.context() as mp:  # pairs not deduplicated
        mp.setattr(np, "unique", lambda a, axis=None: a)
        assert not _point_map_pin()
    orig = P.point_map
    with monkeypatch.context() as mp:  # sides swapped
        mp.setattr(P, "point_map", lambda prob, x: orig(_Elems(prob.vn, prob.vm), x))
        assert not _point_map_pin()
    with monkeypatch.context() as mp:  # first corner only
        mp.setattr(P, "point_map", lambda prob, x: orig(_Elems(prob.vm[:, :1], prob.vn[:, :1]), x))
        assert not _point_map_pin()
