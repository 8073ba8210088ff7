"""Pins of the oracle's neighbour lists (Sect. 2.2: particles within h):
a library k-d tree on tie-free data, symmetry, exact ties."""
import numpy as np
from scipy.spatial import cKDTree

import oracle


def test_neighbours_match_kdtree():
    rng = np.random.default_rng(21)
    pos = rng.normal(size=(4000, 3)) * 0.2
    h = 0.03
    off, idx = oracle.neighbours(pos, h)
    tree = cKDTree(pos)
    # skip rows with a pair within 1e-9 of the radius (rounding ties)
    d, _ = tree.query(pos, k=60, distance_upper_bound=h * 1.0001)
    amb = np.any(np.abs(d - h) < 1e-9, axis=1)
    lists = tree.query_ball_point(pos, r=h)
    checked = 0
    for i in range(pos.shape[0]):
        if amb[i]:
            continue
        ref = sorted(j for j in lists[i] if j != i)
        assert list(idx[off[i]:off[i + 1]]) == ref
        checked += 1
    assert checked > 3900
    assert off[-1] > 4000  # non-trivial lists


def test_neighbours_symmetric_and_rows():
    rng = np.random.default_rng(22)
    pos = rng.uniform(size=(1500, 3))
    off, idx = oracle.neighbours(pos, 0.05)
    pairs = {(i, int(j)) for i in range(1500) for j in idx[off[i]:off[i + 1]]}
    assert all((j, i) in pairs for (i, j) in pairs)
    assert all(i != j for (i, j) in pairs)
    rows = np.array([7, 3, 1499])
    o2, i2 = oracle.neighbours(pos, 0.05, rows=rows)
    for r, i in enumerate(rows):
        assert np.array_equal(i2[o2[r]:o2[r + 1]], idx[off[i]:off[i + 1]])


def test_neighbour_ties_and_coincidence():
    h = 0.5  # exactly representable; h*h = 0.25 exactly
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.0, 0.0],
                    [0.0, 0.3, 0.4], [0.0, -0.3, 0.39999]])
    off, idx = oracle.neighbours(pos, h)
    rows = [list(idx[off[i]:off[i + 1]]) for i in range(5)]
    assert rows[0] == [2, 4]  # r = h exactly excluded; coincident kept
    assert rows[1] == []
    assert rows[2] == [0, 4]
    assert rows[3] == []      # (0, 0.3, 0.4): r^2 rounds to 0.25 = h^2
    assert rows[4] == [0, 2]
    assert oracle.is_neighbour(pos[0], pos[2], h)
    assert not oracle.is_neighbour(pos[0], pos[0] + [0.5, 0, 0], h)
