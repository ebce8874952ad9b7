"""Slab decomposition over two processes (gloo, CPU): the plan, the halo exchange and the
collectives of paper_1507_06767_gb300/partition.py, with the FP64 oracle as each rank's step.
Each rank steps its slab plus one ghost plane per neighbour; after every step the crossing
populations of the boundary planes go to the neighbours.  The owned planes must equal the
single-domain oracle bit for bit (every cell's update reads only its pull sources), the local
block maxima and the all-gathered top-fraction flags must equal the single-domain ones, and the
all-reduced mass and momentum must match to round-off."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from tests import seeded

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


CASES = {
    # name: (q, nx, ny, nz, periodic, block, steps)
    "d3q19_walls": (19, 12, 10, 32, 0, 8, 12),
    "d3q19_periodic_z": (19, 10, 12, 24, O.PERIODIC_Z, 8, 12),
    "d2q9_lid": (9, 24, 32, 1, 0, 8, 30),
}


def initial(q, shape, seed):
    c, w, _ = O.lattice(q)
    return w[:, None, None, None] * (1.0 + seeded.relative_perturbation(seed, (q,) + shape, 0.02))


def single_domain(case):
    q, nx, ny, nz, per, block, steps = CASES[case]
    o = O.Oracle(q, nx, ny, nz, 0.6, lid=(0.05, 0.0, 0.0), periodic=per)
    f = initial(q, (nz, ny, nx), 77)
    K = None
    for _ in range(steps):
        f, K, _, _ = o.step(f, sensor=True)
    return f, K


def rank_main(rank, world, port, case, out):
    from paper_1507_06767_gb300 import partition as PT

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q, nx, ny, nz, per, block, steps = CASES[case]
        axis_n = nz if q == 19 else ny
        slab_periodic = bool(per & (O.PERIODIC_Z if q == 19 else O.PERIODIC_Y))
        slabs = PT.plan(axis_n, world, block, slab_periodic)
        me = slabs[rank]
        lo_g = 1 if me.below is not None else 0
        hi_g = 1 if me.above is not None else 0
        f_full = initial(q, (nz, ny, nx), 77)
        # the slab axis is array axis 1 (z) for D3Q19; for D2Q9 move y there
        if q == 9:
            f_full = f_full.transpose(0, 2, 1, 3)  # (q, y, 1, x)
        sel = [(p % axis_n) for p in range(me.lo - lo_g, me.hi + hi_g)]
        f_ext = torch.from_numpy(np.ascontiguousarray(f_full[:, sel]))
        n_ext = f_ext.shape[1]
        # the oracle sees the extended slab as a lattice with walls at its ends along the slab
        # axis; the ghost planes' own updates are wrong and are overwritten by the next exchange
        per_local = per & ~(O.PERIODIC_Z if q == 19 else O.PERIODIC_Y)
        if q == 19:
            o = O.Oracle(q, nx, ny, n_ext, 0.6, lid=(0.05, 0.0, 0.0), periodic=per_local)
        else:
            o = O.Oracle(q, nx, n_ext, 1, 0.6, lid=(0.05, 0.0, 0.0), periodic=per_local)
        K = None
        for _ in range(steps):
            if q == 19:
                f_np, K, _, _ = o.step(f_ext.numpy(), sensor=True)
                f_ext = torch.from_numpy(f_np)
            else:
                f_np, K, _, _ = o.step(f_ext.numpy().transpose(0, 2, 1, 3), sensor=True)
                f_ext = torch.from_numpy(np.ascontiguousarray(f_np.transpose(0, 2, 1, 3)))
                K = K.transpose(1, 0, 2)
            PT.exchange_halos(f_ext, q, me)
        own = f_ext[:, lo_g:n_ext - hi_g].numpy()
        Kown = K[lo_g:n_ext - hi_g]
        # local block maxima (cuts fall on block edges), then the global ones in block order
        if q == 19:
            bm = O.block_max(Kown, block)
        else:
            bm = O.block_max(Kown.transpose(1, 0, 2)[0], block)
        allm = PT.gather_maxima(torch.from_numpy(bm)).numpy()
        # mass and momentum of the owned planes, summed over the ranks
        own_o = O.Oracle(q, nx, ny if q == 19 else (me.hi - me.lo), (me.hi - me.lo) if q == 19
                         else 1, 0.6)
        own_arr = own if q == 19 else np.ascontiguousarray(own.transpose(0, 2, 1, 3))
        m, j = own_o.conservation(own_arr)
        sums = PT.allreduce_sums(torch.tensor([m] + list(j), dtype=torch.float64))
        out[rank] = (me.lo, me.hi, own, bm, allm, sums.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_rank_slabs_match_single_domain(case):
    q, nx, ny, nz, per, block, steps = CASES[case]
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, case, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    f_ref, K_ref = single_domain(case)
    if q == 9:
        f_ref = f_ref.transpose(0, 2, 1, 3)
    parts = [out[r] for r in range(2)]
    for lo, hi, own, bm, allm, sums in parts:
        assert np.array_equal(own, f_ref[:, lo:hi]), (lo, hi)
    # block maxima: the ranks' maxima in rank order are the single-domain maxima
    ref_bm = O.block_max(K_ref if q == 19 else K_ref[0], block)
    assert np.array_equal(parts[0][4], ref_bm) and np.array_equal(parts[1][4], ref_bm)
    assert np.array_equal(O.flags_top(parts[0][4], 0.25), O.flags_top(ref_bm, 0.25))
    o = O.Oracle(q, nx, ny, nz, 0.6)
    m, j = o.conservation(f_ref if q == 19 else np.ascontiguousarray(f_ref.transpose(0, 2, 1, 3)))
    ref = np.array([m] + list(j))
    # different summation order: round-off of sums of ~N terms of size ~w_i
    for part in parts:
        assert np.allclose(part[5], ref, rtol=0, atol=1e-12 * ref[0])


def test_plan_and_crossing_sets():
    from paper_1507_06767_gb300 import partition as PT

    s = PT.plan(256, 4, 16, periodic=False)
    assert [(x.lo, x.hi) for x in s] == [(0, 64), (64, 128), (128, 192), (192, 256)]
    assert s[0].below is None and s[-1].above is None and s[1].below == 0 and s[1].above == 2
    s = PT.plan(40, 3, 8, periodic=True)  # 5 blocks: 2, 2, 1
    assert [(x.lo, x.hi) for x in s] == [(0, 16), (16, 32), (32, 40)]
    assert s[0].below == 2 and s[2].above == 0
    with pytest.raises(ValueError):
        PT.plan(16, 3, 8, periodic=False)
    for q, axis in ((9, 1), (19, 2)):
        c, _, _ = O.lattice(q)
        assert list(PT.slab_velocity(q)) == c[:, axis].tolist()
        up, down = PT.crossing(q)
        assert len(up) == len(down) == (3 if q == 9 else 5)


# ------------------------------------------------------------------ the CUDA library as the step
# Each slab is a library handle whose cut faces have halos (lbm_set_halo); the crossing populations
# of the boundary planes travel as raw storage bytes (lbm_halo_export / lbm_halo_import).  With
# the one-cell kernel on both sides every cell's update reads the same bytes as in the
# single-domain run, so the slabs must equal it bit for bit, sensor maxima included.
GPU_CASES = {
    # name: (q, nx, ny, nz, periodic, dtype, slabs, steps)
    "d3q19_f32_walls_3": (19, 20, 18, 40, 0, "F32", 3, 25),
    "d3q19_f16s_ragged_2": (19, 17, 12, 33, O.PERIODIC_X, "F16S", 2, 20),
    "d3q19_f64_periodic_z_2": (19, 12, 10, 24, O.PERIODIC_Z | O.PERIODIC_Y, "F64", 2, 15),
    "d3q19_bf16s_periodic_z_1": (19, 16, 9, 16, O.PERIODIC_Z, "BF16S", 1, 10),
    "d2q9_f32_lid_3": (9, 40, 32, 1, 0, "F32", 3, 60),
    "d2q9_f64_periodic_y_2": (9, 24, 24, 1, O.PERIODIC_X | O.PERIODIC_Y, "F64", 2, 40),
}


def _lib():
    torch_ = pytest.importorskip("torch")
    if not torch_.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1507_06767_gb300 as pkg

    return pkg


def _slab_setup(L, case, slab, f0):
    q, nx, ny, nz, per, dtype, _, _ = GPU_CASES[case]
    from paper_1507_06767_gb300 import partition as PT

    axis_bit = O.PERIODIC_Z if q == 19 else O.PERIODIC_Y
    n_loc = slab.hi - slab.lo
    dims = (nx, ny, n_loc) if q == 19 else (nx, n_loc, 1)
    lat = L.Lattice(q, *dims, 0.6, dtype=getattr(L, "LBM_" + dtype), lid=(0.05, 0.0),
                    periodic=per & ~axis_bit)
    L.lbm_set_kernel_variant(lat.h, L.LBM_KERNEL_CELL)
    L.lbm_set_sensor_every(lat.h, 1)
    lat.set_halo(PT.halo_faces(slab))
    part = f0[:, slab.lo:slab.hi] if q == 19 else f0[:, :, slab.lo:slab.hi]
    lat.set_populations(np.ascontiguousarray(part))
    return lat


def _reference_run(L, case, f0):
    q, nx, ny, nz, per, dtype, _, steps = GPU_CASES[case]
    ref = L.Lattice(q, nx, ny, nz, 0.6, dtype=getattr(L, "LBM_" + dtype), lid=(0.05, 0.0),
                    periodic=per)
    L.lbm_set_kernel_variant(ref.h, L.LBM_KERNEL_CELL)
    L.lbm_set_sensor_every(ref.h, 1)
    ref.set_populations(f0)
    ref.step(steps)
    out = ref.populations(), ref.sensor(8)
    ref.close()
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("device_messages", [False, True])
@pytest.mark.parametrize("case", sorted(GPU_CASES))
def test_library_slabs_match_single_domain(case, device_messages):
    """All slabs of the plan in one process, the exchange emulated between steps: host messages,
    or device messages (CUDA tensors, asynchronous on each handle's stream)."""
    L = _lib()
    import torch as T
    from paper_1507_06767_gb300 import partition as PT

    q, nx, ny, nz, per, dtype, nslab, steps = GPU_CASES[case]
    axis_bit = O.PERIODIC_Z if q == 19 else O.PERIODIC_Y
    n_slow = nz if q == 19 else ny
    f0 = initial(q, (nz, ny, nx), 1507)
    slabs = PT.plan(n_slow, nslab, 8, bool(per & axis_bit))
    lats = [_slab_setup(L, case, s, f0) for s in slabs]
    elems, nbytes = L.lbm_halo_size(lats[0].h)
    assert elems == (5 * nx * ny if q == 19 else 3 * nx)
    for _ in range(steps):
        msgs = {}
        for s, lat in zip(slabs, lats):
            for face, key in ((L.LBM_HALO_HI, "up"), (L.LBM_HALO_LO, "down")):
                if (face == L.LBM_HALO_HI and s.above is None) or \
                        (face == L.LBM_HALO_LO and s.below is None):
                    continue
                if device_messages:
                    buf = T.empty(nbytes, dtype=T.uint8, device="cuda")
                    L.lbm_halo_export(lat.h, face, buf)
                else:
                    buf = lat.halo_export(face)
                msgs[(s.rank, key)] = buf
        for s, lat in zip(slabs, lats):
            # the low halo takes what the slab below sent up, the high one what the slab above
            # sent down
            for face, src in ((L.LBM_HALO_LO, (s.below, "up")), (L.LBM_HALO_HI, (s.above, "down"))):
                if src[0] is None:
                    continue
                if device_messages:
                    L.lbm_halo_import(lat.h, face, msgs[src])
                else:
                    lat.halo_import(face, msgs[src])
        for lat in lats:
            lat.step(1)
    f_ref, bm_ref = _reference_run(L, case, f0)
    got = [lat.populations() for lat in lats]
    bms = [lat.sensor(8) for lat in lats]
    for lat in lats:
        lat.close()
    for s, g in zip(slabs, got):
        want = f_ref[:, s.lo:s.hi] if q == 19 else f_ref[:, :, s.lo:s.hi]
        assert np.array_equal(g, want), (case, s)
    assert np.array_equal(np.concatenate(bms), bm_ref)


@pytest.mark.gpu
def test_halo_arguments_are_checked():
    L = _lib()
    lat = L.Lattice(19, 8, 8, 16, 0.6, periodic=O.PERIODIC_Z)
    with pytest.raises(L.LbmError):  # the slab axis is periodic
        lat.set_halo(L.LBM_HALO_LO)
    L.lbm_set_periodic(lat.h, 0)
    lat.set_halo(L.LBM_HALO_LO)
    with pytest.raises(L.LbmError):  # no halo on the high face
        lat.halo_export(L.LBM_HALO_HI)
    with pytest.raises(L.LbmError):  # periodic slab axis with halos
        L.lbm_set_periodic(lat.h, O.PERIODIC_Z)
    with pytest.raises(L.LbmError):  # only the one-cell kernel takes halos
        L.lbm_set_kernel_variant(lat.h, L.LBM_KERNEL_PAIR)
    with pytest.raises(ValueError):
        lat.halo_import(L.LBM_HALO_LO, np.zeros(3, np.uint8))
    with pytest.raises(L.LbmError):
        L.lbm_set_halo(lat.h, 4)
    lat.close()



def library_rank_main(rank, world, port, case, outdir):
    from paper_1507_06767_gb300 import partition as PT

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = _lib()
        q, nx, ny, nz, per, dtype, _, steps = GPU_CASES[case]
        axis_bit = O.PERIODIC_Z if q == 19 else O.PERIODIC_Y
        n_slow = nz if q == 19 else ny
        f0 = initial(q, (nz, ny, nx), 1507)
        slabs = PT.plan(n_slow, world, 8, bool(per & axis_bit))
        me = slabs[rank]
        lat = _slab_setup(L, case, me, f0)
        for _ in range(steps):
            PT.exchange_lattice_halos(lat, me)
            lat.step(1)
        bm = lat.sensor(8)
        allm = PT.gather_maxima(torch.from_numpy(bm)).numpy()
        m, j = lat.conservation()
        sums = PT.allreduce_sums(torch.tensor([m] + list(j), dtype=torch.float64))
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), lo=me.lo, hi=me.hi,
                 f=lat.populations(), allm=allm, sums=sums.numpy())
        lat.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["d3q19_f32_walls_3", "d3q19_f64_periodic_z_2", "d2q9_f32_lid_3"])
def test_two_rank_library_slabs_match_single_domain(case, tmp_path):
    """Two processes (gloo, host-staged halos through partition.exchange_lattice_halos), both on
    the one GPU: their kernels never wait on each other, the exchange happens between steps on the
    host.  Owned populations, all-gathered block maxima and all-reduced sums against the
    single-domain library run."""
    L = _lib()
    q, nx, ny, nz, per, dtype, _, steps = GPU_CASES[case]
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=library_rank_main, args=(r, 2, port, case, str(tmp_path)))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    f0 = initial(q, (nz, ny, nx), 1507)
    f_ref, bm_ref = _reference_run(L, case, f0)
    ref = L.Lattice(q, nx, ny, nz, 0.6, dtype=getattr(L, "LBM_" + dtype), periodic=per)
    ref.set_populations(f_ref)
    m, j = ref.conservation()
    ref.close()
    for r in range(2):
        d = np.load(tmp_path / f"rank{r}.npz")
        lo, hi = int(d["lo"]), int(d["hi"])
        want = f_ref[:, lo:hi] if q == 19 else f_ref[:, :, lo:hi]
        assert np.array_equal(d["f"], want), r
        assert np.array_equal(d["allm"], bm_ref), r
        assert np.allclose(d["sums"], [m] + list(j), rtol=0, atol=1e-12 * m)
