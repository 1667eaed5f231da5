"""Coarse-to-fine candidates (Sec. 4): the host library's mask equals the oracle's (boolean
ring-matrix powers) bit for bit; with no rings it is exactly the mapped coarse pairs; with one
ring around the coarse ground truth it contains every fine ground-truth pair (a midpoint
vertex is one edge from both ends of its coarse edge on either mesh)."""
import numpy as np
import pytest

from oracle import problem as P
from synth import instances as I


@pytest.fixture(scope="module")
def lib():
    from paper_2310_08230_gb300.build import build

    build()
    from paper_2310_08230_gb300 import api

    return api


@pytest.fixture(scope="module")
def pair():
    return I.coarse_fine_pair(2)


def _gt_pairs(coarse):
    return np.stack([np.arange(coarse.X.nv), coarse.perm], axis=1)


@pytest.mark.parametrize("rings", [0, 1, 2])
def test_mask_matches_oracle(lib, pair, rings):
    coarse, fine, cx, cy = pair
    rng = np.random.default_rng(rings)
    pairs = np.concatenate([_gt_pairs(coarse),
                            np.stack([rng.integers(0, coarse.X.nv, 10), rng.integers(0, coarse.Y.nv, 10)], 1)])
    got = lib.candidates_coarse_to_fine(pairs, cx, cy, rings, fine.X.T, fine.X.nv, fine.Y.T, fine.Y.nv)
    ref = P.coarse_to_fine_candidates(pairs, cx, cy, rings, fine.X.T, fine.X.nv, fine.Y.T, fine.Y.nv)
    np.testing.assert_array_equal(got.astype(bool), ref)


def test_no_rings_is_the_mapped_pairs(lib, pair):
    coarse, fine, cx, cy = pair
    pairs = _gt_pairs(coarse)
    got = lib.candidates_coarse_to_fine(pairs, cx, cy, 0, fine.X.T, fine.X.nv, fine.Y.T, fine.Y.nv)
    want = np.zeros((fine.X.nv, fine.Y.nv), np.uint8)
    want[cx[pairs[:, 0]], cy[pairs[:, 1]]] = 1
    np.testing.assert_array_equal(got, want)


def test_one_ring_contains_fine_ground_truth(lib, pair):
    coarse, fine, cx, cy = pair
    got = lib.candidates_coarse_to_fine(_gt_pairs(coarse), cx, cy, 1, fine.X.T, fine.X.nv, fine.Y.T, fine.Y.nv)
    assert got[np.arange(fine.X.nv), fine.perm].all()
    assert got.mean() < 0.2  # and prunes most of the product


def test_bad_ids_are_rejected(lib, pair):
    from paper_2310_08230_gb300 import _lib as L

    coarse, fine, cx, cy = pair
    with pytest.raises(L.DiscoError):
        lib.candidates_coarse_to_fine(np.array([[coarse.X.nv, 0]]), cx, cy, 1, fine.X.T, fine.X.nv, fine.Y.T,
                                      fine.Y.nv)
