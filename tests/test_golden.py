"""Printed values of the paper as fixtures: Table I (tests/golden/)."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_table_i():
    rows = []
    with open(os.path.join(GOLDEN, "table1_tetrahedra.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    a = np.array(rows)
    assert a.shape == (6, 5) and np.array_equal(a[:, 0], np.arange(1, 7))
    return a[:, 1:]


def corner_offset(c):
    """(dx, dy, dz) of corner label c = 1 + dx + 2 dy + 4 dz."""
    c -= 1
    return np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], dtype=float)


def test_oracle_uses_table_i():
    assert np.array_equal(oracle.table_i(), load_table_i())


def test_table_i_partitions_the_cube():
    """With the corner labelling c = 1 + dx + 2 dy + 4 dz every tetrahedron of
    Table I has volume 1/6, all share the cube diagonal from corner 3 to 6, and
    every point of the cube lies in exactly one of them (seeded samples)."""
    tab = load_table_i()
    verts = np.array([[corner_offset(c) for c in row] for row in tab])   # (6, 4, 3)
    vols = np.abs(np.linalg.det(verts[:, 1:] - verts[:, :1])) / 6.0
    np.testing.assert_allclose(vols, 1.0 / 6.0, rtol=0, atol=1e-15)
    assert all(3 in row and 6 in row for row in tab)
    pts = np.random.default_rng(1).uniform(0.0, 1.0, (4000, 3))
    inside = np.zeros((6, len(pts)), dtype=bool)
    for t in range(6):
        A = np.vstack([verts[t].T, np.ones(4)])          # barycentric system
        lam = np.linalg.solve(A, np.vstack([pts.T, np.ones(len(pts))]))
        inside[t] = np.all(lam >= -1e-12, axis=0)
    assert np.all(inside.sum(axis=0) == 1)


def test_table_i_distinct_corners_and_pairs():
    """Each tetrahedron has four distinct corners, and the three face-sharing
    pairs the kernels walk together, (1,2), (3,5) and (4,6) in table order,
    share exactly three corners each."""
    tab = load_table_i()
    assert all(len(set(row)) == 4 for row in tab)
    for a, b in ((0, 1), (2, 4), (3, 5)):
        assert len(set(tab[a]) & set(tab[b])) == 3
