"""Pins of the oracle's brute-force neighbor search (Sec. 2.5.1) against
two independent constructions: explicit enumeration of the 27 periodic
images, and scipy's k-d tree."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle.neighbors import (check_box, minimum_image, neighbor_pairs,
                              neighbor_pairs_images, neighbor_rows)
from paper_2402_17660_gb300 import synth

RC = 5.0


def _as_set(i, j):
    return set(zip(i.tolist(), j.tolist()))


def _pbc_edge_case(seed, L=(10.5, 11.0, 12.25), n=40):
    rng = np.random.default_rng(seed)
    L = np.array(L)
    pos = rng.uniform(-0.5, 1.5, (n, 3)) * L          # many atoms outside [0, L)
    pos[0] = [0.0, 0.0, 0.0]                          # on a corner
    pos[1] = [L[0] - 1e-3, L[1] - 1e-3, L[2] - 1e-3]  # across the corner image
    pos[2] = [L[0], 0.5 * L[1], 0.0]                  # exactly on a face
    pos[3] = [-L[0] + 0.7, -2 * L[1] + 0.3, 3 * L[2] + 0.2]  # far image near the corner
    box = np.diag(L)[None]
    return pos.astype(np.float32), np.zeros(n, np.int32), box.astype(np.float32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pbc_matches_image_enumeration(seed):
    pos, batch, box = _pbc_edge_case(seed)
    a = _as_set(*neighbor_pairs(pos, batch, box, RC))
    b = _as_set(*neighbor_pairs_images(pos, batch, box, RC))
    assert a == b and len(a) > 0


def test_batched_pbc_boxes_match_image_enumeration():
    parts = [_pbc_edge_case(s, L=(10.5 + s, 10.6, 11.0 + 0.5 * s), n=15) for s in range(3)]
    pos = np.concatenate([p[0] for p in parts])
    batch = np.concatenate([np.full(15, s, np.int32) for s in range(3)])
    box = np.concatenate([p[2] for p in parts])
    a = _as_set(*neighbor_pairs(pos, batch, box, RC))
    b = _as_set(*neighbor_pairs_images(pos, batch, box, RC))
    assert a == b
    i, j = neighbor_pairs(pos, batch, box, RC)
    assert np.all(batch[i] == batch[j])


def test_no_pbc_matches_kdtree():
    s = synth.random_cluster(200, seed=3)
    i, j = neighbor_pairs(s.pos, s.batch, None, RC)
    t = cKDTree(s.pos.astype(np.float64))
    ref = t.query_pairs(RC, output_type="ndarray")
    ref = {(a, b) for a, b in ref.tolist()} | {(b, a) for a, b in ref.tolist()}
    assert _as_set(i, j) == ref


def test_pbc_matches_periodic_kdtree():
    s = synth.water_box(4, 12.416, seed=7)
    L = s.meta["L"]
    i, j = neighbor_pairs(s.pos, s.batch, s.box, RC)
    p = np.mod(s.pos.astype(np.float64), L)
    t = cKDTree(p, boxsize=L)
    ref = t.query_pairs(RC, output_type="ndarray")
    ref = {(a, b) for a, b in ref.tolist()} | {(b, a) for a, b in ref.tolist()}
    assert _as_set(i, j) == ref


def test_symmetric_sorted_no_self():
    s = synth.water_box(4, 12.416, seed=8)
    i, j = neighbor_pairs(s.pos, s.batch, s.box, RC)
    assert np.all(i != j)
    assert _as_set(i, j) == _as_set(j, i)
    key = i * len(s.z) + j
    assert np.all(np.diff(key) > 0)


def test_rows_match_pairs():
    s = synth.random_cluster(64, seed=11)
    i, j = neighbor_pairs(s.pos, s.batch, None, RC)
    rows = neighbor_rows(s.pos, s.batch, None, RC, range(64))
    for a in range(64):
        assert np.array_equal(rows[a], j[i == a])


def test_minimum_image_is_nearest():
    rng = np.random.default_rng(4)
    B = np.diag([10.0, 11.0, 12.0])
    r = rng.uniform(-40, 40, (500, 3))
    m = minimum_image(r, B)
    assert np.all(np.abs(m) <= np.diag(B) / 2 + 1e-12)
    shifts = np.round((r - m) @ np.linalg.inv(B))
    assert np.allclose((r - m) @ np.linalg.inv(B), shifts)


def test_box_too_small_rejected():
    with pytest.raises(ValueError):
        check_box(np.diag([9.9, 20.0, 20.0]), RC)
    with pytest.raises(ValueError):
        check_box(np.array([[10.0, 0, 0], [1.0, 12.0, 0.5], [0, 0, 12.0]]), RC)


def test_generated_inputs_keep_margin():
    for s, radii in ((synth.small_molecule(0), (5.0,)), (synth.water_box(10, 31.04, seed=1), (5.0,))):
        i, j = neighbor_pairs(s.pos, s.batch, s.box, 5.0 + 1e-3)
        r = s.pos.astype(np.float64)[i] - s.pos.astype(np.float64)[j]
        if s.box is not None:
            r = minimum_image(r, s.box[0])
        d = np.linalg.norm(r, axis=1)
        for R in radii:
            assert np.all(np.abs(d - R) >= 1e-4)


# ---------------------------------------------------------------- triclinic
TRICLINIC_BOXES = [
    np.array([[12.0, 0, 0], [3.6, 11.5, 0], [2.4, -2.9, 12.2]]),      # reduced tilts
    np.array([[20.0, 0, 0], [14.0, 13.0, 0], [-9.0, 8.0, 13.0]]),     # not reduced, widths >= 2 rc
]


def _tri_cloud(seed, B, n=48):
    rng = np.random.default_rng(seed)
    frac = rng.uniform(-0.5, 1.5, (n, 3))             # many atoms outside the cell
    pos = frac @ B
    pos[0] = 0.0
    pos[1] = B[0] + B[1] + B[2] - 1e-3                 # across the far corner
    return pos.astype(np.float32), np.zeros(n, np.int32), B.astype(np.float32)[None]


@pytest.mark.parametrize("k", range(len(TRICLINIC_BOXES)))
@pytest.mark.parametrize("seed", [0, 1])
def test_triclinic_pbc_matches_image_enumeration(k, seed):
    """The sequential c, b, a reduction against brute force over 125 images,
    on a reduced and a strongly tilted (not reduced) cell."""
    pos, batch, box = _tri_cloud(seed, TRICLINIC_BOXES[k])
    a = _as_set(*neighbor_pairs(pos, batch, box, RC))
    b = _as_set(*neighbor_pairs_images(pos, batch, box, RC, reach=2))
    assert a == b and len(a) > 0


def test_triclinic_minimum_image_is_nearest():
    """For pair vectors whose nearest image is within the cutoff, the
    reduction returns that image (brute force over 125 images)."""
    B = TRICLINIC_BOXES[1]
    rng = np.random.default_rng(5)
    near = rng.uniform(-1, 1, (2000, 3))
    near *= (rng.uniform(0, RC, 2000) / np.linalg.norm(near, axis=1))[:, None]
    n = rng.integers(-3, 4, (2000, 3))
    r = near + n @ B
    got = minimum_image(r, B)
    assert np.allclose(got, near, atol=1e-9)


def test_lattice_equivalent_triclinic_cell_gives_the_same_pairs():
    """The cube of side L and the cell a = (L,0,0), b = (L,L,0), c = (0,L,L)
    span the same lattice (a unimodular change of basis); with all widths
    >= 2 rc the pair sets and the nearest-image vectors coincide."""
    s = synth.water_box(6, 18.6, seed=3)
    L = 18.6
    cube = s.box
    skew = np.array([[[L, 0, 0], [L, L, 0], [0, L, L]]], np.float32)
    ia, ja = neighbor_pairs(s.pos, s.batch, cube, RC)
    ib, jb = neighbor_pairs(s.pos, s.batch, skew, RC)
    assert np.array_equal(ia, ib) and np.array_equal(ja, jb)
    p = s.pos.astype(np.float64)
    assert np.allclose(minimum_image(p[ia] - p[ja], cube[0]), minimum_image(p[ib] - p[jb], skew[0]), atol=1e-9)


def test_triclinic_box_too_narrow_rejected():
    L = 17.0                                            # widths L, L/sqrt(2), L/sqrt(3) < 2 rc
    with pytest.raises(ValueError):
        check_box(np.array([[L, 0, 0], [L, L, 0], [0, L, L]]), RC)

