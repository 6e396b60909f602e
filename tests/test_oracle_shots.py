"""Pins of the oracle's shot count (Sec. II-C.3, minimum rectangle partition): shapes
whose minimum is known by inspection (a rectangle, an L, a plus, a frame, a staircase,
a checkerboard), the count of separate pieces, and invariance under the symmetries of
the square (the search order is row-major, the answer must not be)."""
import numpy as np
import pytest

from oracle import shots


def grid(rows):
    return np.array([[c == "#" for c in r] for r in rows], dtype=np.uint8)


@pytest.mark.parametrize("rows,expected", [
    (["###", "###"], 1),
    (["#..", "#..", "###"], 2),                        # L
    ([".#.", "###", ".#."], 3),                        # plus
    (["####", "#..#", "####"], 4),                     # frame around a hole
    (["#...", "##..", "###.", "####"], 4),             # staircase
    (["#.#", ".#.", "#.#"], 5),                        # checkerboard: one per pixel
    (["##..", "##..", "..##", "..##"], 2),             # two squares touching at a corner
    (["#####", "#...#", "#.#.#", "#...#", "#####"], 5),  # frame with an island
    (["", ], 0),
])
def test_known_minima(rows, expected):
    M = grid(rows) if rows != [""] else np.zeros((2, 2), np.uint8)
    assert shots.min_partition(M) == expected


def test_symmetry_invariance():
    rng = np.random.default_rng(0)
    for _ in range(25):
        M = (rng.random((4, 5)) < 0.55).astype(np.uint8)
        v = shots.min_partition(M)
        for T in (M.T, M[::-1], M[:, ::-1], M[::-1, ::-1].T):
            assert shots.min_partition(np.ascontiguousarray(T)) == v


def test_pieces_add():
    a = grid(["##.", "#..", "..."])
    b = grid(["...", "...", ".##"])
    assert shots.min_partition(a | b) == shots.min_partition(a) + shots.min_partition(b)
