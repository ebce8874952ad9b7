"""GPU parity of the multi-level block mesh (lbm_blocks_step, FP32) with the FP64 oracle
(oracle/lbm_multilevel.c), through the C ABI.

Tolerances: populations max|f_gpu - f_ref| / max|f_ref| <= 2e-6 after 12 cycles of a 3-level
lid-driven mesh (FP32 rounding of f, interpolation and restriction add a few roundings per cycle);
block sensor maxima 1e-4 relative (K is a mean of |f^neq| / f^eq with f^neq ~ 1e-4 f).
"""
import numpy as np
import pytest

import oracle as O

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


def three_level_leaf():
    leaf = np.ones((4, 3, 3), np.int8)
    leaf[0, :, :] = 0
    leaf[2, 2, 1] = 2  # next to the lid plane (y = top)
    leaf[2, 1, 1] = 2
    return leaf


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    m = ~np.isnan(b)
    return float(np.abs(a[m] - b[m]).max() / np.abs(b[m]).max())


@pytest.mark.parametrize("graphs", [True, False])
def test_three_level_cavity_matches_oracle(L, graphs):
    leaf = three_level_leaf()
    edge, lmax, tau, cycles = 8, 2, 0.6, 12
    g = L.BlockMesh(leaf, edge, lmax, tau, lid=(0.1, 0.02), graphs=graphs)
    o = O.MultiLevel(leaf, edge, lmax, tau, lid=(0.1, 0.0, 0.02))
    for level in range(lmax + 1):
        n, tau_l, nblocks, threads, cpt, _ = g.info(level)
        assert (n, nblocks) == (o.level_info(level)[0], int((leaf >= level).sum()))
        assert abs(tau_l - o.level_info(level)[1]) < 1e-15
        assert threads in (128, 256, 512) and cpt >= 1 and cpt & (cpt - 1) == 0
    bm = g.step(cycles, block_max=True)
    o.cycles(cycles)
    for level in range(lmax + 1):
        assert rel(g.leaf_field(level), o.leaf_field(level)) < 2e-6, level
    ref = o.block_max()
    assert rel(bm, ref) < 1e-4
    g.close()


FORM_APPLIES = {"FLAT": (0, lambda n: True), "TILED": (1, lambda n: n in (8, 16, 32, 64)),
                "SELECT": (2, lambda n: n in (16, 32, 64)), "PAIR": (3, lambda n: n in (8, 16, 32, 64))}


@pytest.mark.parametrize("form,periodic", [(f, 0) for f in FORM_APPLIES] +
                         [("SELECT", "XZ"), ("PAIR", "XZ")])
def test_step_forms_match_oracle(L, form, periodic):
    """Every form of the level step kernel, forced on the levels whose block edge it applies to,
    against the FP64 oracle: a 3-level mesh with 4 / 8 / 16 cells per block edge, where the face
    lanes and face rows of the finest level meet a same-level neighbour, an interpolated ghost and
    a wall, and the finest blocks touch the moving lid; with periodic x and z axes the neighbours
    across the domain's x and z faces are the wrapped blocks."""
    leaf = three_level_leaf()
    leaf[2, 2, 2] = 2  # an x-neighbour on the finest level, at the x wall
    edge, lmax, tau, cycles = 16, 2, 0.6, 6
    per = (L.LBM_PERIODIC_X | L.LBM_PERIODIC_Z) if periodic else 0
    g = L.BlockMesh(leaf, edge, lmax, tau, lid=(0.1, 0.02), periodic=per,
                    step_form=getattr(L, "LBM_STEP_FORM_" + form))
    want, applies = FORM_APPLIES[form]
    for level in range(lmax + 1):
        n = g.info(level)[0]
        if applies(n):
            assert g.schedule(level)[0] == want, level
    o = O.MultiLevel(leaf, edge, lmax, tau, lid=(0.1, 0.0, 0.02),
                     periodic=(O.PERIODIC_X | O.PERIODIC_Z) if periodic else 0)
    bm = g.step(cycles, block_max=True)
    o.cycles(cycles)
    for level in range(lmax + 1):
        assert rel(g.leaf_field(level), o.leaf_field(level)) < 2e-6, level
    assert rel(bm, o.block_max()) < 1e-4
    g.close()


@pytest.mark.parametrize("schedule", ["GRAPH", "PERSISTENT"])
def test_graph_replay_is_bitwise_direct_launches(L, schedule):
    """Replaying a cycle from its captured graph gives the same bits as launching it directly.
    The step form, the restriction and the schedule are fixed, so that both builds run the same
    arithmetic (the autotuner may otherwise pick different forms in the two builds)."""
    leaf = three_level_leaf()
    out = []
    for graphs in (True, False):
        g = L.BlockMesh(leaf, 8, 2, 0.6, lid=(0.1, 0.0), graphs=graphs,
                        step_form=L.LBM_STEP_FORM_PAIR, fusion=L.LBM_FUSION_SEPARATE,
                        schedule=getattr(L, "LBM_SCHEDULE_" + schedule))
        g.step(5)
        out.append([g.leaf_field(level) for level in range(3)])
        g.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b, equal_nan=True)


def test_couette_across_interface_on_gpu(L):
    """The Couette pin of the oracle, on the GPU: linear profile across a level interface."""
    U, D = 0.01, 16.0
    leaf = np.zeros((1, 4, 1), np.int8)
    leaf[:, 2:, :] = 1
    g = L.BlockMesh(leaf, 4, 1, 0.8, lid=(U, 0.0), periodic=L.LBM_PERIODIC_X | L.LBM_PERIODIC_Z)
    g.step(6000)
    for level, lo, hi in ((0, 0.0, 8.0), (1, 8.0, 16.0)):
        f = g.leaf_field(level)
        with np.errstate(invalid="ignore"):
            ux = (f[[1, 7, 9, 11, 13]].sum(0) - f[[2, 8, 10, 12, 14]].sum(0)) / f.sum(0)
        h = 2 ** (1 - level)
        y = (np.arange(ux.shape[1]) + 0.5) * h
        sel = (y > lo) & (y < hi)
        prof = np.array([np.nanmean(ux[:, j, :]) for j in np.where(sel)[0]])
        assert np.abs(prof - U * y[sel] / D).max() < 2e-4 * U
    g.close()


def test_single_level_mesh_matches_uniform_path(L):
    """With one level the block mesh is the uniform lattice: it follows the uniform fused step to
    FP32 rounding (different kernels, same arithmetic)."""
    leaf = np.zeros((2, 2, 3), np.int8)
    g = L.BlockMesh(leaf, 8, 0, 0.7, lid=(0.1, 0.0))
    g.step(20)
    u = L.Lattice(L.LBM_D3Q19, 24, 16, 16, 0.7, dtype=L.LBM_F32, lid=(0.1, 0.0))
    u.step(20)
    assert rel(g.leaf_field(0), u.populations()) < 1e-6
    g.close()
    u.close()


def test_block_mesh_argument_errors(L):
    h = L.lbm_create(L.LBM_D3Q19, 24, 8, 8, 0.6)
    try:
        bad = np.array([2, 0, 0], np.int8)  # a level-2 block touching level 0
        with pytest.raises(L.LbmError) as ei:
            L.lbm_blocks_step(h, L.LevelBatch(3, 1, 1, 8, 2, bad.ctypes.data, 1, None))
        assert ei.value.status == L.LBM_EINVAL
        ok = np.zeros(3, np.int8)
        with pytest.raises(L.LbmError) as ei:  # 3 x 4 != 24
            L.lbm_blocks_step(h, L.LevelBatch(3, 1, 1, 4, 0, ok.ctypes.data, 1, None))
        assert ei.value.status == L.LBM_EINVAL
        with pytest.raises(L.LbmError) as ei:
            L.lbm_blocks_get(h, 0, 0, np.empty(1))
        assert ei.value.status == L.LBM_ESTATE
        for form in (-1, L.LBM_STEP_FORM_PAIR + 1):
            with pytest.raises(L.LbmError) as ei:
                L.lbm_blocks_set_step_form(h, form)
            assert ei.value.status == L.LBM_EINVAL
        for mode in (-1, L.LBM_SCHEDULE_PERSISTENT_LEAN + 1):
            with pytest.raises(L.LbmError) as ei:
                L.lbm_blocks_set_schedule(h, mode)
            assert ei.value.status == L.LBM_EINVAL
    finally:
        L.lbm_destroy(h)


def test_bench_mesh_full_size_one_cycle(L):
    """The multi-level benchmark mesh at full size (16^3 blocks of 32 finest cells, 512^3 finest,
    3 levels; 4096 / 1408 / 336 blocks at levels 0 / 1 / 2), in its benchmark launch configuration
    (autotuned shapes, graph replay): every block of every level set to a seeded perturbed state,
    one cycle on the GPU and in the FP64 oracle, every block of every level compared (2e-6, as
    above; FP32 storage of the seeded state is a 6e-8 relative difference of the inputs)."""
    import bench
    from tests import seeded

    w = bench.WORKLOADS["d3q19_blocks_512_3level"]
    leaf = bench.block_placement(w, L)
    tau = bench.tau_of(w)
    g = L.BlockMesh(leaf, w["block"], w["lmax"], tau, lid=(w["u"], 0.0))
    g.step(0)  # builds the mesh (and autotunes) at rest
    o = O.MultiLevel(leaf, w["block"], w["lmax"], tau, lid=(w["u"], 0.0, 0.0))
    _, wts, _ = O.lattice(19)
    rng = seeded.rng(4096)
    flat = leaf.reshape(-1)
    for level in range(w["lmax"] + 1):
        n = g.info(level)[0]
        for b in np.where(flat >= level)[0]:
            f = wts[:, None, None, None] * (1.0 + rng.uniform(-0.01, 0.01, size=(19, n, n, n)))
            g.set_block(level, int(b), f)
            o.set_block(level, int(b), f)
    g.step(1)
    o.cycles(1)
    worst = 0.0
    for level in range(w["lmax"] + 1):
        for b in np.where(flat >= level)[0]:
            ref = o.get_block(level, int(b))
            worst = max(worst, float(np.abs(g.get_block(level, int(b)) - ref).max() /
                                     np.abs(ref).max()))
    assert worst < 2e-6, worst
    g.close()


@pytest.mark.parametrize("fusion", ["SEPARATE", "FUSED", "BRICK"])
def test_fused_restriction_matches_oracle(L, fusion):
    """A 2-level mesh whose finest blocks have 16 cells per edge, with the restriction onto level 0
    as a separate kernel and fused into the finest level's second sub-step (tiled form, brick
    form): each against the FP64 oracle after 10 cycles (the fused forms sum the 8 fine cells in
    other orders)."""
    leaf = np.zeros((3, 3, 4), np.int8)
    leaf[1, 2, 1:3] = 1
    leaf[2, 2, 2] = 1
    edge, lmax, tau, cycles = 16, 1, 0.6, 10
    g = L.BlockMesh(leaf, edge, lmax, tau, lid=(0.1, 0.02),
                    fusion=getattr(L, "LBM_FUSION_" + fusion))
    assert g.schedule(1)[2] == {"SEPARATE": 0, "FUSED": 4, "BRICK": 1}[fusion]
    o = O.MultiLevel(leaf, edge, lmax, tau, lid=(0.1, 0.0, 0.02))
    bm = g.step(cycles, block_max=True)
    o.cycles(cycles)
    for level in range(lmax + 1):
        assert rel(g.leaf_field(level), o.leaf_field(level)) < 2e-6, level
    assert rel(bm, o.block_max()) < 1e-4
    g.close()


@pytest.mark.parametrize("edge", [16, 32])
def test_brick_restriction_three_levels(L, edge):
    """The brick form of the fused restriction on the 3-level lid-driven mesh (finest blocks of 8
    and 16 cells per edge: with 8, every brick touches a block face; the x-face lanes select their
    neighbour), with graph replay, against the FP64 oracle after 8 cycles."""
    leaf = three_level_leaf()
    lmax, tau, cycles = 2, 0.6, 8
    g = L.BlockMesh(leaf, edge // 2, lmax, tau, lid=(0.1, 0.02), fusion=L.LBM_FUSION_BRICK)
    assert g.schedule(2)[2] == 1
    o = O.MultiLevel(leaf, edge // 2, lmax, tau, lid=(0.1, 0.0, 0.02))
    bm = g.step(cycles, block_max=True)
    o.cycles(cycles)
    for level in range(lmax + 1):
        assert rel(g.leaf_field(level), o.leaf_field(level)) < 2e-6, level
    assert rel(bm, o.block_max()) < 1e-4
    g.close()


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("fusion,schedule", [("SEPARATE", "PERSISTENT"),
                                             ("BRICK", "PERSISTENT_BRICK"),
                                             ("BRICK", "PERSISTENT_LEAN")])
def test_persistent_cycle_matches_oracle(L, graphs, fusion, schedule):
    """One persistent launch per cycle: the cycle's ghost fills, level steps and restrictions as
    tasks of one kernel, ordered by device-side counters; the kernel with the finest level's brick
    phases and the lean one (plain steps and restriction phases), each forced.  The 3-level
    lid-driven mesh (finest blocks of 16 cells, so the brick form applies) against the FP64 oracle
    after 10 cycles, replayed from a captured graph and launched directly."""
    leaf = three_level_leaf()
    edge, lmax, tau, cycles = 16, 2, 0.6, 10
    g = L.BlockMesh(leaf, edge, lmax, tau, lid=(0.1, 0.02), graphs=graphs,
                    fusion=getattr(L, "LBM_FUSION_" + fusion),
                    schedule=getattr(L, "LBM_SCHEDULE_" + schedule))
    assert g.cycle_form() == L.LBM_SCHEDULE_PERSISTENT
    o = O.MultiLevel(leaf, edge, lmax, tau, lid=(0.1, 0.0, 0.02))
    bm = g.step(cycles, block_max=True)
    o.cycles(cycles)
    for level in range(lmax + 1):
        assert rel(g.leaf_field(level), o.leaf_field(level)) < 2e-6, level
    assert rel(bm, o.block_max()) < 1e-4
    g.close()


def test_persistent_cycle_bench_mesh_one_cycle(L):
    """The full-size multi-level benchmark mesh run by the persistent cycle: every block of every
    level from a seeded perturbed state, one cycle, against the FP64 oracle (2e-6)."""
    import bench
    from tests import seeded

    w = bench.WORKLOADS["d3q19_blocks_512_3level"]
    leaf = bench.block_placement(w, L)
    tau = bench.tau_of(w)
    g = L.BlockMesh(leaf, w["block"], w["lmax"], tau, lid=(w["u"], 0.0),
                    schedule=L.LBM_SCHEDULE_PERSISTENT)
    o = O.MultiLevel(leaf, w["block"], w["lmax"], tau, lid=(w["u"], 0.0, 0.0))
    _, wts, _ = O.lattice(19)
    rng = seeded.rng(4097)
    flat = leaf.reshape(-1)
    for level in range(w["lmax"] + 1):
        n = g.info(level)[0]
        for b in np.where(flat >= level)[0]:
            f = wts[:, None, None, None] * (1.0 + rng.uniform(-0.01, 0.01, size=(19, n, n, n)))
            g.set_block(level, int(b), f)
            o.set_block(level, int(b), f)
    g.step(1)
    o.cycles(1)
    worst = 0.0
    for level in range(w["lmax"] + 1):
        for b in np.where(flat >= level)[0]:
            ref = o.get_block(level, int(b))
            worst = max(worst, float(np.abs(g.get_block(level, int(b)) - ref).max() /
                                     np.abs(ref).max()))
    assert worst < 2e-6, worst
    g.close()


def test_persistent_cycle_wait_runs_out(L):
    """A bounded device wait of the persistent cycle that runs out: lbm_debug_hold_copies makes every
    dependency wait unreachable (nothing faults; the waiting CTA gives up after the limit, raises
    the abort flag and every CTA stops claiming tasks), so lbm_blocks_step with block maxima returns
    LBM_ETIMEOUT.  After a rebuild the mesh runs correctly again on the same context."""
    leaf = three_level_leaf()
    edge, lmax, tau = 8, 2, 0.6
    g = L.BlockMesh(leaf, edge, lmax, tau, lid=(0.1, 0.02), schedule=L.LBM_SCHEDULE_PERSISTENT)
    L.lbm_debug_set_wait_limit(g.h, 1_000_000)  # 1 ms
    L.lbm_debug_hold_copies(g.h, 1)
    with pytest.raises(L.LbmError) as ei:
        g.step(1, block_max=True)
    assert ei.value.status == L.LBM_ETIMEOUT
    L.lbm_debug_hold_copies(g.h, 0)
    L.lbm_debug_set_wait_limit(g.h, 0)
    L.lbm_reset(g.h)  # clears the error word
    L.lbm_blocks_set_schedule(g.h, L.LBM_SCHEDULE_PERSISTENT)  # discards the mesh
    bm = g.step(6, block_max=True)  # rebuilt from rest
    o = O.MultiLevel(leaf, edge, lmax, tau, lid=(0.1, 0.0, 0.02))
    o.cycles(6)
    for level in range(lmax + 1):
        assert rel(g.leaf_field(level), o.leaf_field(level)) < 2e-6, level
    assert rel(bm, o.block_max()) < 1e-4
    g.close()
