"""The library's shot count (Sec. II-C.3, minimum rectangle partition; host code, no
GPU needed) against the oracle's exhaustive search on tiny masks: random masks of
several densities (holes, diagonal contacts, islands), and shapes with known minima."""
import numpy as np
import pytest

from oracle import shots


@pytest.fixture(scope="module")
def dv():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_12529_gb300 as dv
    return dv


@pytest.mark.parametrize("density", [0.3, 0.5, 0.7, 0.85])
def test_matches_exhaustive_search_on_random_masks(dv, density):
    rng = np.random.default_rng(int(density * 100))
    for _ in range(60):
        n = int(rng.integers(1, 7))
        M = (rng.random((n, n)) < density).astype(np.uint8)
        assert dv.devel_shot_count(M) == shots.min_partition(M), M


def test_known_shapes(dv):
    frame = np.ones((6, 6), np.uint8)
    frame[2:4, 2:4] = 0
    assert dv.devel_shot_count(frame) == 4
    plus = np.zeros((5, 5), np.uint8)
    plus[2, :] = 1
    plus[:, 2] = 1
    assert dv.devel_shot_count(plus) == 3
    checker = (np.add.outer(np.arange(6), np.arange(6)) % 2).astype(np.uint8)
    assert dv.devel_shot_count(checker) == checker.sum()
    assert dv.devel_shot_count(np.zeros((4, 4), np.uint8)) == 0
    assert dv.devel_shot_count(np.ones((9, 9), np.uint8)) == 1


def test_large_mask_is_fast_and_consistent(dv):
    """A 512^2 mask of many rectangles: the count of disjoint rectangles is exact."""
    rng = np.random.default_rng(3)
    M = np.zeros((512, 512), np.uint8)
    count = 0
    for r in range(0, 500, 25):
        for c in range(0, 500, 25):
            if rng.random() < 0.6:
                h, w = rng.integers(3, 20, 2)
                M[r:r + h, c:c + w] = 1
                count += 1
    assert dv.devel_shot_count(M) == count
