"""GPU parity of lbm_regrid (tag, buffer, proper nesting, Berger-Rigoutsos clustering; Sec. 5.2)
with the numpy oracle (oracle/regrid.py).  Integer work after the tag decision, so the boxes and
tag grids must be identical; both sides take the tag decision (K > T) on the same doubles."""
import numpy as np
import pytest

import oracle as O
from oracle import regrid as R
from tests import seeded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1507_06767_gb300 as pkg

    return pkg


def lattice_for(L, shape, periodic=0):
    nz, ny, nx = shape
    q = L.LBM_D3Q19 if nz > 1 else L.LBM_D2Q9
    return L.Lattice(q, nx, ny, nz, 0.6, dtype=L.LBM_F64, periodic=periodic)


def dev(K):
    import torch

    return torch.from_numpy(np.ascontiguousarray(K, dtype=np.float64)).cuda()


def covered_mask(tshape, seed):
    """The coarser level's coverage: the whole tag grid minus three random boxes."""
    g = seeded.rng(seed)
    allowed = np.ones(tshape, bool)
    for _ in range(3):
        lo = [int(g.integers(0, n)) for n in tshape]
        hi = [min(n, lo_ + int(g.integers(1, max(2, n // 2) + 1))) for lo_, n in zip(lo, tshape)]
        allowed[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = False
    return allowed


CASES = [
    # shape (nz, ny, nx), coarsen, buffer, efficiency, min_width, periodic, nest (None: no mask)
    ((1, 96, 128), 1, 1, 0.8, 1, 0, None),
    ((1, 96, 128), 4, 1, 0.8, 2, 0, None),
    ((1, 97, 131), 2, 2, 0.7, 1, 3, 1),
    ((24, 20, 28), 1, 1, 0.8, 1, 0, None),
    ((24, 20, 28), 2, 1, 0.8, 2, 0, 1),
    ((33, 17, 41), 4, 0, 0.5, 1, 7, None),
    ((32, 32, 32), 1, 2, 1.0, 1, 2, 2),
    ((40, 36, 33), 3, 1, 0.8, 3, 5, 1),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_regrid_matches_oracle(L, case):
    shape, r, b, eff, w, per, nest = CASES[case]
    K = seeded.blob_field(700 + case, shape)
    T = float(np.quantile(K, 0.9))
    allowed = None
    if nest is not None:
        allowed = covered_mask(R.tag_cells(np.zeros(shape), 0.0, r).shape, 800 + case)
    ref_boxes, ref_tags = R.regrid(K, T, coarsen=r, buffer=b, efficiency=eff, min_width=w,
                                   allowed=allowed, nest=nest or 0, periodic=per)
    lat = lattice_for(L, shape, per)
    boxes, tags = lat.regrid(T, coarsen=r, buffer=b, efficiency=eff, min_width=w,
                             allowed=allowed, nest=nest or 0, field=dev(K))
    lat.close()
    assert np.array_equal(tags, ref_tags)
    assert boxes.tolist() == ref_boxes.tolist()
    assert len(ref_boxes) > 1  # the case exercises the clustering


def test_regrid_at_the_bench_lattice_size(L):
    """256^3 sensor-shaped field (the size of the timed D3Q19 lattice), tag cells of 4^3."""
    shape = (256, 256, 256)
    K = seeded.blob_field(901, (64, 64, 64))
    K = np.repeat(np.repeat(np.repeat(K, 4, 0), 4, 1), 4, 2)  # piecewise constant on 4^3
    T = float(np.quantile(K, 0.85))
    ref_boxes, ref_tags = R.regrid(K, T, coarsen=4, buffer=1)
    lat = lattice_for(L, shape)
    boxes, tags = lat.regrid(T, coarsen=4, buffer=1, field=dev(K))
    lat.close()
    assert np.array_equal(tags, ref_tags)
    assert boxes.tolist() == ref_boxes.tolist()


def test_regrid_from_the_cavity_sensor(L):
    """End to end: a D2Q9 FP64 cavity run on the GPU and in the oracle; the regrid of the handle's
    own sensor field equals the oracle's regrid of the oracle's field (no cell within 1e-8 of T,
    far outside the 1e-12 FP64 parity of the sensor)."""
    n, steps = 128, 1500
    tau = O.tau_from_re(0.1, n, 100.0)
    o = O.Oracle(9, n, n, 1, tau, lid=(0.1, 0.0, 0.0))
    _, Kref = o.run(o.rest(), steps, sensor_last=True)
    lat = L.Lattice(L.LBM_D2Q9, n, n, 1, tau, dtype=L.LBM_F64, lid=(0.1, 0.0))
    L.lbm_set_sensor_field(lat.h, 1)
    L.lbm_set_sensor_every(lat.h, 1)
    lat.step(steps)
    Kgpu = lat.sensor_field()
    assert np.abs(Kgpu - Kref).max() <= 1e-10 * np.abs(Kref).max()
    T = 4.0 * (4.0 / 3.0) * tau * 0.1 / n
    assert np.abs(Kref - T).min() > 1e-8 * T
    for r, w in ((1, 2), (4, 1)):
        ref_boxes, ref_tags = R.regrid(Kref, T, coarsen=r, buffer=1, min_width=w)
        boxes, tags = lat.regrid(T, coarsen=r, buffer=1, min_width=w)
        assert np.array_equal(tags, ref_tags)
        assert boxes.tolist() == ref_boxes.tolist()
        assert len(boxes) >= 1
    lat.close()


def test_regrid_edge_cases(L):
    shape = (1, 40, 48)
    lat = lattice_for(L, shape)
    # no tag: no box
    boxes, tags = lat.regrid(1.0, field=dev(np.zeros(shape)))
    assert boxes.shape == (0, 6) and not tags.any()
    # every cell tagged (NaN tags too): one box, the lattice
    K = np.ones(shape)
    K[0, 3, 5] = np.nan
    boxes, tags = lat.regrid(0.5, field=dev(K))
    assert boxes.tolist() == [[0, 0, 0, 48, 40, 1]] and tags.all()
    # a single NaN is tagged (with its buffer)
    K = np.zeros(shape)
    K[0, 10, 20] = np.nan
    boxes, _ = lat.regrid(0.5, field=dev(K))
    assert boxes.tolist() == [[19, 9, 0, 22, 12, 1]]
    # too many boxes for the output: LBM_EINVAL with the count
    K = np.zeros(shape)
    K[0, 5, 5] = K[0, 30, 40] = 1.0
    with pytest.raises(L.LbmError) as ei:
        lat.regrid(0.5, field=dev(K), max_boxes=1)
    assert ei.value.status == L.LBM_EINVAL
    # bad arguments
    for kw in (dict(coarsen=0), dict(buffer=-1), dict(min_width=0), dict(efficiency=1.5),
               dict(efficiency=float("nan")), dict(nest=-1)):
        with pytest.raises(L.LbmError) as ei:
            lat.regrid(0.5, field=dev(K), **kw)
        assert ei.value.status == L.LBM_EINVAL
    # no recorded sensor field
    with pytest.raises(L.LbmError) as ei:
        lat.regrid(0.5)
    assert ei.value.status == L.LBM_ESTATE
    lat.close()


def test_regrid_from_an_fp32_cavity_sensor(L):
    """End to end on an FP32 D3Q19 handle (the FP32 field's 16-byte tag pass, tag cells of 4^3):
    the threshold sits in a gap of the oracle's tag-cell maxima wider than the FP32 sensor error
    (1e-4 relative), so both sides tag the same cells and must build the same boxes."""
    nx, ny, nz, steps = 32, 40, 24, 300
    tau = O.tau_from_re(0.1, ny, 400.0)
    o = O.Oracle(19, nx, ny, nz, tau, lid=(0.1, 0.0, 0.0))
    _, Kref = o.run(o.rest(), steps, sensor_last=True)
    m = Kref.reshape(nz // 4, 4, ny // 4, 4, nx // 4, 4).max(axis=(1, 3, 5)).ravel()
    v = np.unique(m)
    gaps = v[1:] / v[:-1] - 1.0
    lo = int(0.6 * len(v))
    k = lo + int(np.argmax(gaps[lo:int(0.9 * len(v))]))
    assert gaps[k] > 2e-3
    T = float(np.sqrt(v[k] * v[k + 1]))
    lat = L.Lattice(L.LBM_D3Q19, nx, ny, nz, tau, dtype=L.LBM_F32, lid=(0.1, 0.0))
    L.lbm_set_sensor_field(lat.h, 1)
    L.lbm_set_sensor_every(lat.h, 1)
    lat.step(steps)
    ref_boxes, ref_tags = R.regrid(Kref, T, coarsen=4, buffer=1, min_width=2)
    boxes, tags = lat.regrid(T, coarsen=4, buffer=1, min_width=2)
    assert np.array_equal(tags, ref_tags)
    assert boxes.tolist() == ref_boxes.tolist() and len(boxes) >= 1
    lat.close()
