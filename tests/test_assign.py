"""The host step of the re-indexing (gevp_assign_min_cost, the library's Hungarian
method) against brute force on tiny tables and against scipy's assignment solver on
larger ones, including rectangular tables, ties and the near-identity tables that
eigenvectors of consecutive problems give. Runs on the CPU: the call needs no device."""
import itertools

import numpy as np
import pytest


def _cost(c, perm):
    return float(c[np.arange(c.shape[0]), perm].sum())


def _valid(perm, kn):
    return len(set(perm.tolist())) == len(perm) and perm.min() >= 0 and perm.max() < kn


@pytest.mark.parametrize("ko,kn", [(1, 1), (3, 3), (4, 6), (6, 6), (5, 7)])
def test_matches_brute_force(ko, kn):
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(10 * ko + kn)
    for _ in range(20):
        c = rng.uniform(0, 1, (ko, kn))
        if rng.uniform() < 0.3:
            c = np.round(c * 4) / 4   # many ties
        best = min(_cost(c, np.array(p)) for p in itertools.permutations(range(kn), ko))
        perm = gevp.assign_min_cost(c)
        assert _valid(perm, kn)
        assert abs(_cost(c, perm) - best) <= 1e-12


@pytest.mark.parametrize("ko,kn,kind", [(200, 200, "uniform"), (150, 190, "uniform"), (400, 480, "near_identity"),
                                        (300, 300, "blocks")])
def test_matches_scipy(ko, kn, kind):
    from scipy.optimize import linear_sum_assignment
    from paper_1007_4400_gb300 import gevp
    rng = np.random.default_rng(ko + kn)
    if kind == "uniform":
        c = rng.uniform(0, 1, (ko, kn))
    elif kind == "near_identity":
        # 1 - |cosine| of slightly rotated vectors under a permutation: small on one entry per row
        c = 1.0 - np.abs(rng.uniform(0, 0.2, (ko, kn)))
        sh = rng.permutation(kn)[:ko]
        c[np.arange(ko), sh] = rng.uniform(0, 1e-3, ko)
    else:
        # degenerate clusters: equal costs inside 3 x 3 diagonal blocks
        c = np.ones((ko, kn))
        for b in range(0, ko, 3):
            c[b:b + 3, b:b + 3] = 0.5
    r, col = linear_sum_assignment(c)
    perm = gevp.assign_min_cost(c)
    assert _valid(perm, kn)
    assert abs(_cost(c, perm) - float(c[r, col].sum())) <= 1e-9


def test_rejects_bad_input():
    from paper_1007_4400_gb300 import gevp
    with pytest.raises(ValueError):
        gevp.assign_min_cost(np.zeros((3, 2)))
    with pytest.raises(ValueError):
        gevp.assign_min_cost(np.array([[0.0, np.nan]]))
    assert gevp.assign_min_cost(np.zeros((0, 4))).shape == (0,)
