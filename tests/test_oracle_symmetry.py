"""Pins of the oracle's cube-symmetry helpers (oracle/skeleton.py).  The 48
signed permutations of the axes map the n x n face-cell grids of the
directions (Sec. 2.2) onto themselves; cells of one orbit share their
skeletons and M2L operators.  Pinned against: the group axioms, a round trip
through cell centres, the octree's integer direction rule (an independent
implementation) away from cell boundaries, and Burnside's count of the orbits
of the cube group on the face cells."""
import itertools

import numpy as np
import pytest

from oracle import octree as ot
from oracle import skeleton as S


def _matrix(sym):
    return S.apply_sym(sym, np.eye(3)).T     # column k = image of e_k


def test_symmetries_are_the_cube_group():
    mats = [_matrix(s) for s in S.SYMMETRIES]
    assert len(mats) == 48
    keys = {m.astype(int).tobytes() for m in mats}
    assert len(keys) == 48                                   # distinct
    for m in mats:
        assert np.array_equal(m @ m.T, np.eye(3))            # orthogonal, entries 0 / +-1
    for a, b in itertools.product(mats[::5], mats[::7]):
        assert (a @ b).astype(int).tobytes() in keys         # closed under composition
    x = np.array([0.3, -1.7, 2.9])
    for sym, m in zip(S.SYMMETRIES, mats):
        assert np.allclose(S.apply_sym(sym, x), m @ x)       # apply_sym is the linear map


@pytest.mark.parametrize("n", [1, 2, 3, 4, 8])
def test_cell_centres_round_trip(n):
    for c in range(6 * n * n):
        v = S.cell_center_dir(c, n)
        assert np.max(np.abs(v)) == 1.0
        assert S.cell_of_dir(v, n) == c


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_cell_of_dir_matches_the_integer_direction_rule(n):
    rng = np.random.default_rng(n)
    m = rng.integers(-40, 41, size=(4000, 3))
    am = np.abs(m)
    M = am.max(axis=1)
    keep = (M > 0) & ((am == M[:, None]).sum(axis=1) == 1)   # one face axis
    face_axis = np.argmax(am, axis=1)
    for d in range(3):                                        # not on a cell boundary
        on_edge = (n * (m[:, d] + M)) % (2 * np.maximum(M, 1)) == 0
        keep &= (d == face_axis) | ~on_edge
    m = m[keep]
    assert m.shape[0] > 500
    ref = ot.direction(m, n)
    got = np.array([S.cell_of_dir(v.astype(float), n) for v in m])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_orbits_of_face_cells_counted_by_burnside(n):
    """The cube group acts transitively on the 6 faces with the dihedral group
    of the square as a face's stabiliser, so the orbits of face cells are the
    orbits of D4 on the n x n grid: by Burnside, (n^2 + 2n) / 8 for even n
    (only the two diagonal reflections fix cells, n each), 1 for n = 1."""
    canon, which = S.canonical_cells(n)
    nd = 6 * n * n
    reps = np.unique(canon)
    expected = 1 if n == 1 else (n * n + 2 * n) // 8
    assert reps.size == expected
    sizes = np.bincount(np.searchsorted(reps, canon))
    assert sizes.sum() == nd and all(48 % s == 0 for s in sizes)
    for c in range(nd):
        k = canon[c]
        assert k <= c and canon[k] == k
        v = S.apply_sym(S.SYMMETRIES[which[c]], S.cell_center_dir(k, n))
        assert S.cell_of_dir(v, n) == c                       # Q(canonical) = c
