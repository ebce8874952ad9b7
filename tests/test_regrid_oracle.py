"""Pins of the regridding oracle (oracle/regrid.py): tagging, buffer cells, proper nesting and
Berger-Rigoutsos clustering (Sec. 5.2), checked against library morphology, hand-worked cases
and the invariants any valid clustering keeps."""
import numpy as np
import pytest

from oracle import regrid as R
from tests.seeded import rng_for

ndi = pytest.importorskip("scipy.ndimage")


def test_tag_cells_hand_case_ragged_and_nan():
    # 2-D field 3 x 5 (ny, nx), tag cells of 2 x 2: the high column and row are partial
    K = np.zeros((3, 5))
    K[2, 4] = 0.5  # the lone cell of the corner tag cell (1, 2)
    K[0, 1] = 0.1  # exactly T: not tagged (strict >)
    K[1, 2] = np.nan  # tag cell (0, 1)
    t = R.tag_cells(K, 0.1, 2)
    assert t.shape == (1, 2, 3)
    want = np.zeros((1, 2, 3), bool)
    want[0, 1, 2] = True
    want[0, 0, 1] = True
    assert np.array_equal(t, want)
    # r = 1 is the plain comparison
    assert np.array_equal(R.tag_cells(K, 0.1, 1)[0], (K > 0.1) | np.isnan(K))


def test_tag_cells_3d_coarsens_z():
    K = np.zeros((4, 4, 4))
    K[3, 0, 0] = 1.0
    t = R.tag_cells(K, 0.5, 2)
    assert t.shape == (2, 2, 2) and t.sum() == 1 and t[1, 0, 0]


@pytest.mark.parametrize("b", [1, 2])
def test_dilate_is_cube_dilation(b):
    rng = rng_for("regrid-dilate", b)
    tags = rng.random((7, 9, 11)) < 0.03
    ref = ndi.binary_dilation(tags, structure=np.ones((3, 3, 3), bool), iterations=b)
    assert np.array_equal(R.dilate(tags, b), ref)


@pytest.mark.parametrize("periodic", [1, 2, 4, 7])
def test_dilate_periodic_is_dilation_of_the_tiled_grid(periodic):
    rng = rng_for("regrid-dilate-periodic", periodic)
    tags = rng.random((6, 7, 8)) < 0.04
    reps = tuple(3 if periodic & (1 << (2 - ax)) else 1 for ax in range(3))
    tiled = np.tile(tags, reps)
    big = ndi.binary_dilation(tiled, structure=np.ones((3, 3, 3), bool), iterations=1)
    sl = tuple(slice(n, 2 * n) if r == 3 else slice(None) for n, r in zip(tags.shape, reps))
    assert np.array_equal(R.dilate(tags, 1, periodic), big[sl])


@pytest.mark.parametrize("nest", [1, 2])
def test_erode_is_cube_erosion_with_covered_outside(nest):
    rng = rng_for("regrid-erode", nest)
    allowed = ndi.binary_dilation(rng.random((8, 10, 12)) < 0.05,
                                  structure=np.ones((3, 3, 3), bool), iterations=2)
    ref = ndi.binary_erosion(allowed, structure=np.ones((3, 3, 3), bool), iterations=nest,
                             border_value=1)
    assert np.array_equal(R.erode(allowed, nest), ref)


def test_erode_periodic_is_erosion_of_the_tiled_grid():
    rng = rng_for("regrid-erode-periodic", 0)
    allowed = rng.random((6, 7, 8)) < 0.8
    tiled = np.tile(allowed, (1, 3, 3))  # y and x periodic
    big = ndi.binary_erosion(tiled, structure=np.ones((3, 3, 3), bool), border_value=1)
    assert np.array_equal(R.erode(allowed, 1, 1 | 2), big[:, 7:14, 8:16])


def rect(shape, *boxes):
    t = np.zeros(shape, bool)
    for (x0, y0, z0, x1, y1, z1) in boxes:
        t[z0:z1, y0:y1, x0:x1] = True
    return t


def test_cluster_one_rectangle_is_its_bounding_box():
    t = rect((5, 12, 10), (2, 3, 1, 7, 9, 4))
    assert R.cluster(t, 0.8) == [(2, 3, 1, 7, 9, 4)]


def test_cluster_splits_at_the_hole():
    # two slabs separated by empty x slabs 4..6: efficiency 0.5 < 0.8, so the box is cut at a hole
    t = rect((1, 4, 12), (1, 0, 0, 4, 4, 1), (7, 0, 0, 10, 4, 1))
    assert R.cluster(t, 0.8) == [(1, 0, 0, 4, 4, 1), (7, 0, 0, 10, 4, 1)]


def test_cluster_l_shape_splits_at_the_inflection():
    # L: rows y = 0, 1 over x = 0..7 and columns x = 0, 1 over y = 0..7 (28 of 64 cells).
    # Signatures along x and y: 8 8 2 2 2 2 2 2, no hole; second differences -6 6 0 0 0 0: one
    # sign change between slabs 1 and 2 on each axis, strength 12; equal distance to the centre,
    # equal length, so axis x wins: cut at x = 2.  Both pieces are then full rectangles.
    t = rect((1, 8, 8), (0, 0, 0, 8, 2, 1), (0, 0, 0, 2, 8, 1))
    assert R.cluster(t, 0.8) == [(0, 0, 0, 2, 8, 1), (2, 0, 0, 8, 2, 1)]


def test_cluster_checkerboard_bisects():
    # a 4 x 4 checkerboard has flat signatures (2 per slab): no hole, no inflection, so it is
    # bisected.  Width 1 ends at single cells (the 8 tags); width 2 stops at the four 2 x 2 boxes
    # (efficiency 0.5, no admissible split left).
    t = np.zeros((1, 4, 4), bool)
    t[0, ::2, ::2] = True
    t[0, 1::2, 1::2] = True
    ones = R.cluster(t, 0.8, 1)
    assert sorted(ones) == sorted((x, y, 0, x + 1, y + 1, 1) for y in range(4) for x in range(4)
                                  if t[0, y, x])
    assert R.cluster(t, 0.8, 2) == [(0, 0, 0, 2, 2, 1), (2, 0, 0, 4, 2, 1), (0, 2, 0, 2, 4, 1),
                                    (2, 2, 0, 4, 4, 1)]


def test_cluster_efficiency_limits():
    rng = rng_for("regrid-eff", 0)
    t = rng.random((3, 9, 13)) < 0.2
    zs, ys, xs = np.nonzero(t)
    bb = (xs.min(), ys.min(), zs.min(), xs.max() + 1, ys.max() + 1, zs.max() + 1)
    assert R.cluster(t, 0.0) == [tuple(int(v) for v in bb)]
    for b in R.cluster(t, 1.0, 1):
        assert t[b[2]:b[5], b[1]:b[4], b[0]:b[3]].all()


def check_valid(t, boxes, eff, w):
    cover = np.zeros(t.shape, np.int64)
    for (x0, y0, z0, x1, y1, z1) in boxes:
        sub = t[z0:z1, y0:y1, x0:x1]
        cover[z0:z1, y0:y1, x0:x1] += 1
        # tight: every face slab holds a tag
        assert sub[0].any() and sub[-1].any() and sub[:, 0].any() and sub[:, -1].any()
        assert sub[:, :, 0].any() and sub[:, :, -1].any()
        lens = (x1 - x0, y1 - y0, z1 - z0)
        if sub.sum() < eff * sub.size:
            # bisection is admissible whenever an axis is >= 2 w long
            assert all(L < 2 * w for L in lens), "an inefficient box that could still be split"
    assert cover.max() <= 1, "overlapping boxes"
    assert (cover[t] == 1).all(), "uncovered tag"


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("w", [1, 2, 3])
def test_cluster_invariants_on_random_blobs(seed, w):
    rng = rng_for("regrid-blobs", seed, w)
    shape = (1, 40, 48) if seed % 2 else (12, 14, 16)
    t = np.zeros(shape, bool)
    for _ in range(5):
        c = [rng.integers(0, n) for n in shape]
        rad = rng.integers(1, 5)
        zz, yy, xx = np.ogrid[:shape[0], :shape[1], :shape[2]]
        t |= (zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2 <= rad ** 2
    boxes = R.cluster(t, 0.8, w)
    check_valid(t, boxes, 0.8, w)
    # with width 1 every box reaches the efficiency (single cells always can)
    if w == 1:
        for (x0, y0, z0, x1, y1, z1) in boxes:
            sub = t[z0:z1, y0:y1, x0:x1]
            assert sub.sum() >= 0.8 * sub.size


def test_regrid_buffer_and_nesting():
    # one hot cell in an 16 x 16 field; buffer 1 makes it a 3 x 3 box; nesting inside a region
    # that ends next to it cuts the buffer back
    K = np.zeros((16, 16))
    K[5, 9] = 1.0
    boxes, tags = R.regrid(K, 0.5, buffer=1)
    assert boxes.tolist() == [[8, 4, 0, 11, 7, 1]]
    allowed = np.zeros((1, 16, 16), bool)
    allowed[0, :, :11] = True  # covered x < 11: eroded by 1 -> x < 10
    boxes, tags = R.regrid(K, 0.5, buffer=1, allowed=allowed, nest=1)
    assert boxes.tolist() == [[8, 4, 0, 10, 7, 1]]
    # at the physical boundary no nesting buffer is needed
    K2 = np.zeros((16, 16))
    K2[0, 0] = 1.0
    boxes, _ = R.regrid(K2, 0.5, buffer=1, allowed=np.ones((1, 16, 16), bool), nest=1)
    assert boxes.tolist() == [[0, 0, 0, 2, 2, 1]]


def test_regrid_coarsened_boxes_in_lattice_cells():
    K = np.zeros((10, 10, 10))
    K[9, 9, 9] = 1.0  # in the partial tag cell (2, 2, 2) of edge 4
    boxes, tags = R.regrid(K, 0.5, coarsen=4, buffer=0)
    assert tags.shape == (3, 3, 3)
    assert boxes.tolist() == [[8, 8, 8, 10, 10, 10]]


def test_cluster_takes_the_hole_nearest_the_centre():
    # slabs x: A = 0..3, B = 5, C = 9..12 over the full y range (L = 13, 9/13 < 0.8).  Holes at
    # x = 4, 6, 7, 8 have |2p - 13| = 5, 1, 1, 3: the cut is at 6 (tie with 7, lower position).
    # A + B then reach 5/6 >= 0.8 and stay one box; cutting at the first hole (4) would instead
    # leave B + C (5/8) to be cut again into three boxes.
    t = rect((1, 3, 13), (0, 0, 0, 4, 3, 1), (5, 0, 0, 6, 3, 1), (9, 0, 0, 13, 3, 1))
    assert R.cluster(t, 0.8) == [(0, 0, 0, 6, 3, 1), (9, 0, 0, 13, 3, 1)]
