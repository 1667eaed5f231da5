"""The split of a batch into pipelined groups (api.balanced_groups): every pair in exactly one
group, groups in ascending order, loads balanced by the longest-processing-time rule, and the
same split as that rule written out directly (no GPU needed)."""
import numpy as np
import pytest

from paper_2310_08230_gb300.api import balanced_groups


def _lpt(w, g):
    load, members = [0.0] * g, [[] for _ in range(g)]
    for i in sorted(range(len(w)), key=lambda i: -w[i]):
        k = int(np.argmin(load))
        members[k].append(i)
        load[k] += w[i]
    return [sorted(m) for m in members if m]


@pytest.mark.parametrize("n,g", [(1, 2), (5, 2), (64, 2), (64, 3), (64, 8), (3, 8)])
def test_groups_cover_every_pair_once_and_balance(n, g):
    rng = np.random.Generator(np.random.PCG64(n * 31 + g))
    w = list(rng.integers(80, 1536, size=n) * rng.integers(8, 25, size=n))
    groups = balanced_groups(w, g)
    assert len(groups) == min(g, n)
    assert sorted(i for m in groups for i in m) == list(range(n))
    assert all(m == sorted(m) for m in groups)
    assert groups == _lpt(w, min(g, n))
    loads = [sum(w[i] for i in m) for m in groups]
    # LPT: no group exceeds the average by more than the largest single weight
    assert max(loads) <= sum(w) / len(groups) + max(w)


def test_equal_weights_split_evenly():
    groups = balanced_groups([1.0] * 10, 4)
    assert sorted(len(m) for m in groups) == [2, 2, 3, 3]
