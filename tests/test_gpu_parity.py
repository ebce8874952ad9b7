"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (written per test):
* FP64 storage: populations and sensor within 1e-12 / 1e-10 relative (the GPU evaluates the same
  formulas on deviations from the rest state, so only the rounding order differs);
* FP32 storage: populations max|f_gpu - f_ref| / max|f_ref| <= 1e-5 after the run's full step
  count; sensor block maxima <= 1e-4 relative (K is a mean of |f^neq|/f^eq, and f^neq is ~1e-4 of
  f, so FP32 rounding of f costs ~1e-4 of K);
* flags: identical except blocks whose oracle maximum lies within 1e-4 (relative) of a decision
  boundary (T, T/2, or the k-th largest maximum).
"""
import math

import numpy as np
import pytest

import oracle as O
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


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def perturbed(o, seed, amp):
    return o.w[:, None, None, None] * (1.0 + seeded.relative_perturbation(seed, o.shape, amp))


def make(L, q, nx, ny, nz, tau, dtype, lid=(0.1, 0.0, 0.0), periodic=0):
    lat = L.Lattice(q, nx, ny, nz, tau, dtype=dtype, lid=(lid[0], lid[2]), periodic=periodic)
    o = O.Oracle(q, nx, ny, nz, tau, lid=lid, periodic=periodic)
    return lat, o


# ----------------------------------------------------------------------------- configuration 1
def test_cavity_d2q9_fp64_128_re100_full_run(L):
    """D2Q9 lid-driven cavity, 128^2, FP64, Re = 100 (u = 0.1, tau = 0.884), 2000 steps, sensor every
    100 steps reduced to 16^2 block maxima, fixed threshold flags.  The threshold reading is four
    times the Couette-level sensor of the mean lid shear, T = 4 (4/3) tau u / N."""
    N, u, re, steps, every, b = 128, 0.1, 100.0, 2000, 100, 16
    tau = O.tau_from_re(u, N, re)
    T = 4.0 * (4.0 / 3.0) * tau * u / N
    lat, o = make(L, 9, N, N, 1, tau, L.LBM_F64)
    L.lbm_set_sensor_every(lat.h, every)
    lat.block = b
    f_ref = o.rest()
    n_flag_cmp = 0
    for k in range(steps // every):
        lat.step(every)
        f_ref, K = o.run(f_ref, every, sensor_last=True)
        ref_max = O.block_max(K, b)
        gpu_max = lat.sensor(b)
        assert gpu_max.shape == (64,)
        assert rel(gpu_max, ref_max) < 1e-10, k
        flags = lat.flag(T)
        ok, ncmp, _ = O.flags_agree(flags, ref_max, "threshold", T, 1e-4)
        assert ok, k
        n_flag_cmp += ncmp
        top = lat.flag_top(0.1)
        ok, _, _ = O.flags_agree(top, ref_max, "top", 0.1, 1e-4)
        assert ok, k
    assert n_flag_cmp > 0.9 * 64 * (steps // every)
    f_gpu = lat.populations()
    assert rel(f_gpu, f_ref) < 1e-12
    # refine and coarsen both occur at the end: the corners under the lid are hot
    assert (flags == 1).any() and (flags == -1).any()
    lat.close()


def test_cavity_d2q9_fp32_matches_fp64_oracle(L):
    """Same cavity with FP32 storage: the populations stay within 1e-5 of the FP64 oracle after 2000
    steps and the per-cell sensor field within 1e-4 of the oracle's largest value."""
    N, tau, steps = 128, O.tau_from_re(0.1, 128, 100.0), 2000
    lat, o = make(L, 9, N, N, 1, tau, L.LBM_F32)
    L.lbm_set_sensor_field(lat.h, 1)
    lat.step(steps)
    f_ref, K = o.run(o.rest(), steps, sensor_last=True)
    assert rel(lat.populations(), f_ref) < 1e-5
    assert rel(lat.sensor_field()[0], K[0]) < 1e-4
    lat.close()


# ----------------------------------------------------------------------------- configuration 2
def test_cavity_d3q19_fp32_ragged_full_step_count(L):
    """D3Q19 cavity in FP32 at the 256^3 run's tau (0.5768) and lid speed, on a ragged 40x36x33
    lattice (tiles of 8 and blocks of 16 with partial ones at every high end), for the full 10000
    steps; sensor every step, 16^3 block maxima and top-10 % flags."""
    tau, steps = O.tau_from_re(0.1, 256, 1000.0), 10000
    lat, o = make(L, 19, 40, 36, 33, tau, L.LBM_F32)
    L.lbm_set_sensor_every(lat.h, 1)
    lat.step(steps)
    f_ref, K = o.run(o.rest(), steps, sensor_last=True)
    assert rel(lat.populations(), f_ref) < 1e-5
    ref_max = O.block_max(K, 16)
    gpu_max = lat.sensor(16)
    assert gpu_max.shape == (27,)
    assert rel(gpu_max, ref_max) < 1e-4
    ok, _, _ = O.flags_agree(lat.flag_top(0.1, block=16), ref_max, "top", 0.1, 1e-4)
    assert ok
    ok, _, _ = O.flags_agree(lat.flag_top(0.1, block=8), O.block_max(K, 8), "top", 0.1, 1e-4)
    assert ok
    m0 = float(np.sum(o.w)) * 40 * 36 * 33
    m, _ = lat.conservation()
    assert abs(m - m0) / m0 < 1e-6
    lat.close()


def test_cavity_d3q19_256_full_size_sampled(L):
    """The 256^3 D3Q19 FP32 workload in the benchmark's launch configuration (sensor every step):
    one step from a seeded perturbed state, checked on sampled cells (all corners, edges, faces and
    random interior cells) and on the 16^3 block maxima of sampled blocks, each evaluated by the
    oracle one by one."""
    n, tau = 256, O.tau_from_re(0.1, 256, 1000.0)
    q = 19
    lat = L.Lattice(q, n, n, n, tau, dtype=L.LBM_F32, lid=(0.1, 0.0))
    o = O.Oracle(q, n, n, n, tau, lid=(0.1, 0.0, 0.0))
    L.lbm_set_sensor_every(lat.h, 1)
    f0 = perturbed(o, seed=256, amp=0.03).astype(np.float32)
    lat.set_raw(f0.view(np.uint8).reshape(-1))
    lat.step(1)
    out = lat.raw().view(np.float32).reshape(q, -1)
    gmax = lat.sensor(16)
    f0d = f0.astype(np.float64)
    del f0
    g = seeded.rng(7)
    e = np.array([0, 1, 2, n // 2, n - 3, n - 2, n - 1])
    xs, ys, zs = np.meshgrid(e, e, e, indexing="ij")
    cells = ((zs * n + ys) * n + xs).reshape(-1)
    cells = np.concatenate([cells, g.integers(0, n ** 3, size=4000)])
    ref, _ = o.step_cells(f0d, cells)
    got = out[:, cells].T.astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-7
    # sampled 16^3 blocks, including the corner blocks under the lid
    nb = n // 16
    blocks = [0, nb - 1, nb * (nb - 1), nb * nb * nb - 1, nb * nb * (nb - 1) + nb * (nb - 1)]
    blocks += list(g.integers(0, nb ** 3, size=6))
    for bidx in blocks:
        bx, by, bz = bidx % nb, (bidx // nb) % nb, bidx // (nb * nb)
        z, y, x = np.meshgrid(np.arange(16) + 16 * bz, np.arange(16) + 16 * by,
                              np.arange(16) + 16 * bx, indexing="ij")
        bc = ((z * n + y) * n + x).reshape(-1)
        _, K = o.step_cells(f0d, bc)
        assert abs(gmax[bidx] - K.max()) / K.max() < 1e-5, bidx
    lat.close()


def test_cavity_d3q19_256_full_field_150_steps(L):
    """The 256^3 D3Q19 FP32 workload in the benchmark's launch configuration (automatic kernel,
    sensor every step), 150 steps from a seeded perturbed state, against the FP64 oracle stepping
    the whole lattice: every population of every cell (<= 1e-5 relative), every 16^3 block maximum
    of the last step (<= 1e-4), and the top-10 % and fixed-threshold flags of the lattice against
    the oracle's flag rules on the oracle's own maxima (identical outside the 1e-4 band)."""
    n, q, steps = 256, 19, 150
    tau = O.tau_from_re(0.1, n, 1000.0)
    lat = L.Lattice(q, n, n, n, tau, dtype=L.LBM_F32, lid=(0.1, 0.0))
    o = O.Oracle(q, n, n, n, tau, lid=(0.1, 0.0, 0.0))
    L.lbm_set_sensor_every(lat.h, 1)
    f0 = perturbed(o, seed=1507, amp=0.01).astype(np.float32)
    lat.set_raw(f0.view(np.uint8).reshape(-1))
    f0 = f0.astype(np.float64)  # the oracle starts from the same (FP32-rounded) state
    lat.step(steps)
    gmax = lat.sensor(16)
    top = lat.flag_top(0.1, block=16)
    T = 4.0 * (4.0 / 3.0) * tau * 0.1 / n
    thr = lat.flag(T, block=16)
    f_gpu = lat.raw().view(np.float32).reshape(q, n, n, n)
    lat.close()
    f_ref, K = o.run(f0, steps, sensor_last=True)
    del f0
    scale = np.abs(f_ref).max()
    worst = 0.0
    for i in range(q):  # one direction at a time keeps the host memory in check
        worst = max(worst, float(np.abs(f_gpu[i].astype(np.float64) - f_ref[i]).max()))
    assert worst / scale <= 1e-5, f"populations differ by {worst / scale:.3e} of max|f|"
    ref_max = O.block_max(K, 16)
    assert gmax.shape == (4096,)
    assert rel(gmax, ref_max) <= 1e-4
    ok, ncmp, _ = O.flags_agree(top, ref_max, "top", 0.1, 1e-4)
    assert ok and ncmp >= 4000
    ok, ncmp, _ = O.flags_agree(thr, ref_max, "threshold", T, 1e-4)
    assert ok and ncmp >= 4000
    # the top-10 % rule refines exactly ceil(0.1 * 4096) = 410 blocks
    assert int((top == 1).sum()) == 410 and int((top == 0).sum()) == 4096 - 410


# ----------------------------------------------------------------------------- edge cases
EDGE_CASES = [
    (9, (1, 1, 1), 0), (9, (2, 3, 1), 0), (9, (5, 7, 1), O.PERIODIC_X), (9, (33, 17, 1), 0),
    (9, (9, 8, 1), O.PERIODIC_X | O.PERIODIC_Y), (19, (1, 1, 1), 0), (19, (2, 3, 2), 0),
    (19, (5, 7, 3), O.PERIODIC_Z), (19, (33, 17, 9), 0), (19, (8, 8, 8), 7),
    (19, (31, 9, 17), O.PERIODIC_X | O.PERIODIC_Y),
]


@pytest.mark.parametrize("q,dims,periodic", EDGE_CASES)
@pytest.mark.parametrize("dtype", ["F64", "F32"])
def test_edge_lattices_perturbed(L, q, dims, periodic, dtype):
    """Tiny and ragged lattices where most cells touch a wall, every periodic combination, seeded
    perturbed states, a lid with x and z components: populations, per-cell sensor and 8-tile maxima
    after 5 steps."""
    dt = getattr(L, "LBM_" + dtype)
    lid = (0.08, 0.0, 0.03 if q == 19 else 0.0)
    lat, o = make(L, q, *dims, tau=0.71, dtype=dt, lid=lid, periodic=periodic)
    L.lbm_set_sensor_field(lat.h, 1)
    f0 = perturbed(o, seed=sum(dims) * q + periodic, amp=0.03)
    lat.set_populations(f0)
    f_in = lat.populations()  # the storage-rounded input (exact for FP64)
    if dtype == "F64":
        assert np.array_equal(f_in, f0)
    lat.step(5)
    f_ref, K = o.run(f_in, 5, sensor_last=True)
    tol_f, tol_k = (1e-13, 1e-11) if dtype == "F64" else (2e-6, 1e-4)
    assert rel(lat.populations(), f_ref) < tol_f
    assert rel(lat.sensor_field(), K) < tol_k
    assert rel(lat.sensor(8), O.block_max(K, 8)) < tol_k
    # moments of the stored post-collision state (collision keeps them: Eqs. rho, u)
    rho, u = lat.moments()
    _, rho_ref, u_ref = o.sensor(f_ref)
    assert np.abs(rho - rho_ref).max() < (1e-14 if dtype == "F64" else 1e-6)
    assert np.abs(u - u_ref).max() < (1e-14 if dtype == "F64" else 1e-6)
    lat.close()


def test_uniform_equilibrium_gpu(L):
    """Eq. (sensor) at f = f_eq: the GPU sensor of a uniform periodic flow is zero to round-off."""
    for q, dims in ((9, (16, 8, 1)), (19, (8, 8, 8))):
        o = O.Oracle(q, *dims, tau=0.8, periodic=7)
        u0 = np.array([0.05, -0.02, 0.03 if q == 19 else 0.0])[:, None, None, None]
        for dt, tol in ((L.LBM_F64, 1e-14), (L.LBM_F32, 2e-6)):
            lat = L.Lattice(q, *dims, 0.8, dtype=dt, lid=(0, 0), periodic=7)
            lat.set_populations(o.equilibrium(1.0, u0))
            L.lbm_set_sensor_every(lat.h, 1)
            lat.step(3)
            assert lat.sensor(8).max() < tol
            lat.close()


# ----------------------------------------------------------------------------- flag builder
@pytest.mark.parametrize("n", [1, 7, 410, 4096, 100003])
@pytest.mark.parametrize("mdtype", ["F32", "F64"])
def test_flag_builder_bit_exact(L, n, mdtype):
    """The flag builder on seeded block maxima with ties, NaNs and values on and one ulp around T and
    T/2: bit-identical to the oracle's rules (both decide in double on the same values)."""
    import torch

    T = 1e-3
    m = seeded.block_maxima(n, n, ties=n // 5, nans=max(0, n // 50), near=(T, n // 10))
    if mdtype == "F64":
        m = m.astype(np.float64)
    dev = torch.from_numpy(m).cuda()
    out = torch.empty(n, dtype=torch.int8, device="cuda")
    dt = getattr(L, "LBM_" + mdtype)
    s = torch.cuda.current_stream().cuda_stream
    L.lbm_flags_from_maxima(dev, dt, n, L.LBM_FLAG_THRESHOLD, T, out, s)
    assert np.array_equal(out.cpu().numpy(), O.flags_threshold(m, T))
    for frac in (0.0, 0.1, 0.5, 1.0, 1.0 / n):
        L.lbm_flags_from_maxima(dev, dt, n, L.LBM_FLAG_TOP, frac, out, s)
        assert np.array_equal(out.cpu().numpy(), O.flags_top(m, frac)), frac


# ----------------------------------------------------------------------------- state handling
def test_checkpoint_resume_and_graphs_bitwise(L):
    """Raw checkpoint + resume continues bit for bit; graph replay gives the same bits as launches."""
    tau = 0.6
    a = L.Lattice(19, 24, 20, 18, tau, dtype=L.LBM_F32)
    a.step(37)
    snap = a.raw()
    a.step(41)
    ref = a.raw()
    b = L.Lattice(19, 24, 20, 18, tau, dtype=L.LBM_F32)
    b.set_raw(snap)
    L.lbm_set_graphs(b.h, 0)
    b.step(41)
    assert np.array_equal(b.raw(), ref)
    a.close()
    b.close()


def test_nan_is_detected_and_refined(L):
    """A NaN planted in the populations makes the FP64 conservation check fail with LBM_ENUMERIC and
    poisons its block's sensor maximum, which the flag rules refine."""
    o = O.Oracle(19, 16, 16, 16, 0.7, lid=(0.1, 0, 0))
    lat = L.Lattice(19, 16, 16, 16, 0.7, dtype=L.LBM_F32)
    f = o.rest()
    f[5, 3, 4, 12] = np.nan  # cell (x=12, y=4, z=3): 8-tile (1, 0, 0)
    lat.set_populations(f)
    with pytest.raises(L.LbmError) as ei:
        lat.conservation()
    assert ei.value.status == L.LBM_ENUMERIC
    L.lbm_set_sensor_every(lat.h, 1)
    lat.step(1)
    m8 = lat.sensor(8)
    assert np.isnan(m8).sum() >= 1
    flags = lat.flag(1.0, block=8)
    assert (flags[np.isnan(m8)] == 1).all()
    lat.close()


def test_sensor_before_any_sensor_step(L):
    lat = L.Lattice(9, 16, 16, 1, 0.7, dtype=L.LBM_F32)
    with pytest.raises(L.LbmError) as ei:
        lat.sensor(8)
    assert ei.value.status == L.LBM_ESTATE
    L.lbm_set_sensor_every(lat.h, 3)
    lat.step(2)
    with pytest.raises(L.LbmError):
        lat.sensor(8)
    lat.step(1)
    assert lat.sensor(8).shape == (4,)
    lat.close()


def test_library_owned_buffers_and_streams(L):
    """Without torch buffers the library allocates its own; work on a side torch stream is ordered
    on that stream."""
    import torch

    o = O.Oracle(19, 12, 10, 9, 0.65, lid=(0.1, 0, 0))
    s = torch.cuda.Stream()
    lat = L.Lattice(19, 12, 10, 9, 0.65, dtype=L.LBM_F64, torch_buffers=False, stream=s)
    lat.step(20)
    f_ref, _ = o.run(o.rest(), 20)
    assert rel(lat.populations(), f_ref) < 1e-13
    lat.close()


def test_profiling_counts_launches(L):
    lat = L.Lattice(19, 32, 32, 32, 0.6, dtype=L.LBM_F32)
    L.lbm_set_profiling(lat.h, 1)
    lat.step(7)
    ms, n = L.lbm_kernel_time(lat.h)
    assert n == 7 and ms > 0
    lat.close()


# ----------------------------------------------------------------------------- kernel variants
STORAGE_TOL = {  # populations (max|df|/max|f| after 3 steps), sensor field (relative to max K)
    "F32": (2e-6, 1e-4),
    "F16S": (1e-4, 2e-3),
    "BF16S": (1e-3, 2e-2),
}


@pytest.mark.parametrize("dtype", ["F32", "F16S", "BF16S"])
@pytest.mark.parametrize("q,dims,periodic", [(19, (40, 20, 18), 0), (19, (48, 12, 10), O.PERIODIC_Z),
                                             (19, (64, 9, 17), O.PERIODIC_X | O.PERIODIC_Y),
                                             (19, (264, 10, 9), O.PERIODIC_X),
                                             (19, (288, 9, 11), 0),
                                             (9, (66, 30, 1), 0)])
def test_kernel_variants_match_oracle(L, dtype, q, dims, periodic):
    """The one-cell kernel, the two-cell packed kernel, the TMA-staged kernel and (16-bit storage)
    the TMA-staged two-cell kernel compute the same step: each matches the oracle from the same
    storage-rounded input within the storage type's tolerance, and they agree with each other to a
    few FP32 roundings.  The lattices are ragged against the TMA work units (256 x 1 x 8 and
    64 x 8 x 8 cells) in every direction.  Shifted FP16 / BF16 storage
    (f - w_i) rounds the deviation from rest to 11 / 8 significant bits per step; the tolerances
    above are those roundings over 3 steps."""
    dt = getattr(L, "LBM_" + dtype)
    lid = (0.1, 0.0, 0.02 if q == 19 else 0.0)
    o = O.Oracle(q, *dims, tau=0.6, lid=lid, periodic=periodic)
    f0 = perturbed(o, seed=77 + q + dims[0], amp=0.02)
    variants = [L.LBM_KERNEL_CELL, L.LBM_KERNEL_PAIR] + ([L.LBM_KERNEL_TMA] if q == 19 else [])
    if q == 19 and dtype != "F32" and dims[0] % 8 == 0:
        variants.append(L.LBM_KERNEL_TMA_PAIR)
    res = {}
    for variant in variants:
        lat = L.Lattice(q, *dims, 0.6, dtype=dt, lid=(lid[0], lid[2]), periodic=periodic)
        L.lbm_set_kernel_variant(lat.h, variant)
        L.lbm_set_sensor_field(lat.h, 1)
        lat.set_populations(f0)
        f_in = lat.populations()
        lat.step(3)
        res[variant] = (f_in, lat.populations(), lat.sensor_field(), lat.sensor(8))
        lat.close()
    tol_f, tol_k = STORAGE_TOL[dtype]
    f_in = res[L.LBM_KERNEL_CELL][0]
    for v in variants:
        assert np.array_equal(f_in, res[v][0])
    f_ref, K = o.run(f_in, 3, sensor_last=True)
    for variant, (_, f, k, m) in res.items():
        assert rel(f, f_ref) < tol_f, variant
        assert rel(k, K) < tol_k, variant
        assert rel(m, O.block_max(K, 8)) < tol_k, variant
    for v in variants[1:]:
        assert rel(res[v][1], res[L.LBM_KERNEL_CELL][1]) < tol_f, v



@pytest.mark.parametrize("dtype", ["F32", "F16S", "BF16S"])
@pytest.mark.parametrize("q,dims,periodic", [(19, (2, 5, 4), 0), (19, (2, 4, 5), O.PERIODIC_X),
                                             (19, (4, 3, 3), O.PERIODIC_X | O.PERIODIC_Z),
                                             (19, (6, 2, 3), 0), (9, (2, 7, 1), 0),
                                             (9, (4, 2, 1), O.PERIODIC_X)])
def test_two_cell_kernel_tiny_lattices(L, dtype, q, dims, periodic):
    """The two-cell kernel on the smallest lattices it takes: nx = 2 puts both x faces in one
    lane (the address-select path serves both of its cells), ny or nz below 3 leaves no interior
    row (every row takes the per-cell gather).  Against the oracle from the same storage-rounded
    input, within the storage type's tolerance, and against the one-cell kernel."""
    dt = getattr(L, "LBM_" + dtype)
    lid = (0.1, 0.0, 0.02 if q == 19 else 0.0)
    o = O.Oracle(q, *dims, tau=0.6, lid=lid, periodic=periodic)
    f0 = perturbed(o, seed=91 + q + dims[1], amp=0.02)
    res = {}
    for variant in (L.LBM_KERNEL_CELL, L.LBM_KERNEL_PAIR):
        lat = L.Lattice(q, *dims, 0.6, dtype=dt, lid=(lid[0], lid[2]), periodic=periodic)
        L.lbm_set_kernel_variant(lat.h, variant)
        L.lbm_set_sensor_field(lat.h, 1)
        lat.set_populations(f0)
        f_in = lat.populations()
        lat.step(3)
        res[variant] = (f_in, lat.populations(), lat.sensor_field())
        lat.close()
    tol_f, tol_k = STORAGE_TOL[dtype]
    f_in = res[L.LBM_KERNEL_CELL][0]
    assert np.array_equal(f_in, res[L.LBM_KERNEL_PAIR][0])
    f_ref, K = o.run(f_in, 3, sensor_last=True)
    for variant, (_, f, k) in res.items():
        assert rel(f, f_ref) < tol_f, variant
        assert rel(k, K) < tol_k, variant
    assert rel(res[L.LBM_KERNEL_PAIR][1], res[L.LBM_KERNEL_CELL][1]) < tol_f


@pytest.mark.parametrize("dtype", ["F16S", "BF16S"])
@pytest.mark.parametrize("dims,periodic", [((8, 8, 8), 0), ((16, 5, 3), O.PERIODIC_X),
                                           ((72, 20, 19), O.PERIODIC_X | O.PERIODIC_Z),
                                           ((136, 17, 23), 0), ((64, 64, 64), 7),
                                           ((200, 12, 9), O.PERIODIC_Y)])
def test_tma_pair_kernel_bitwise_equals_two_cell_kernel(L, dtype, dims, periodic):
    """The TMA-staged two-cell kernel evaluates the same floating-point operations as the two-cell
    kernel on the same stored inputs (the same rows take the packed relaxation, the same rows the
    per-cell gather), so over 50 steps -- mixed sensor and plain steps, graph replay, a lid with x
    and z components -- the stored populations and the sensor maxima are identical bit for bit.
    The lattices cover one tile holding both x faces (nx = 8), x-periodic wrap at both faces,
    partial units in every direction, and fewer rows or planes than a unit."""
    dt = getattr(L, "LBM_" + dtype)
    o = O.Oracle(19, *dims, tau=0.58, lid=(0.09, 0.0, 0.03), periodic=periodic)
    f0 = perturbed(o, seed=311 + sum(dims), amp=0.02)
    out = {}
    for variant in (L.LBM_KERNEL_PAIR, L.LBM_KERNEL_TMA_PAIR):
        lat = L.Lattice(19, *dims, 0.58, dtype=dt, lid=(0.09, 0.03), periodic=periodic)
        L.lbm_set_kernel_variant(lat.h, variant)
        L.lbm_set_sensor_every(lat.h, 7)
        lat.set_populations(f0)
        lat.step(50)
        out[variant] = (lat.raw(), lat.sensor(8))
        lat.close()
    a, b = out[L.LBM_KERNEL_PAIR], out[L.LBM_KERNEL_TMA_PAIR]
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


def test_kernel_variant_applicability(L):
    """A variant that does not apply is refused when it is set (LBM_EINVAL), before any buffer is
    allocated: the two-cell kernel with FP64 storage, an odd nx, or (q + 1) * cells >= 2^32 (its
    32-bit offsets); the TMA kernel on D2Q9; the TMA two-cell kernel with FP32 storage, nx not a
    multiple of 8, 20 * cells >= 2^32, or D2Q9."""
    cases = [(19, (33, 8, 8), "F32", "PAIR"), (19, (32, 8, 8), "F64", "PAIR"),
             (19, (1024, 1024, 208), "F16S", "PAIR"), (9, (64, 64, 1), "F32", "TMA"),
             (19, (64, 8, 8), "F32", "TMA_PAIR"), (19, (36, 8, 8), "F16S", "TMA_PAIR"),
             (19, (1024, 1024, 208), "BF16S", "TMA_PAIR"), (9, (64, 64, 1), "F16S", "TMA_PAIR")]
    for q, (nx, ny, nz), dt, variant in cases:
        h = L.lbm_create(q, nx, ny, nz, 0.6)
        try:
            L.lbm_set_dtype(h, getattr(L, "LBM_" + dt))
            with pytest.raises(L.LbmError) as ei:
                L.lbm_set_kernel_variant(h, getattr(L, "LBM_KERNEL_" + variant))
            assert ei.value.status == L.LBM_EINVAL, (q, nx, dt, variant)
            L.lbm_set_kernel_variant(h, L.LBM_KERNEL_CELL)  # always applies
        finally:
            L.lbm_destroy(h)


def test_tma_kernel_long_run_and_sensor_steps(L):
    """The TMA kernel over many steps with mixed sensor / non-sensor steps and graph replay, on a
    lattice with several work units per CTA and an odd plane count per unit: it follows the
    one-cell kernel to FP32 rounding (the two evaluate the same formulas in a different order)."""
    dims, tau = (64, 40, 35), 0.58
    out = {}
    for variant in (L.LBM_KERNEL_CELL, L.LBM_KERNEL_TMA):
        lat = L.Lattice(19, *dims, tau, dtype=L.LBM_F32)
        L.lbm_set_kernel_variant(lat.h, variant)
        L.lbm_set_sensor_every(lat.h, 7)
        lat.step(50)
        out[variant] = (lat.raw(), lat.sensor(8), lat.sensor(16))
        lat.close()
    a, b = out[L.LBM_KERNEL_CELL], out[L.LBM_KERNEL_TMA]
    fa, fb = a[0].view(np.float32), b[0].view(np.float32)
    assert rel(fb, fa) < 1e-5
    assert rel(b[1], a[1]) < 1e-4 and rel(b[2], a[2]) < 1e-4


# ----------------------------------------------------------------------------- level map
@pytest.mark.parametrize("q,dims,dtype,kband", [(9, (128, 128, 1), "F64", 1e-10),
                                               (19, (40, 36, 33), "F32", 2e-4)])
def test_levels_and_time_average(L, q, dims, dtype, kband):
    """Sec. 3.4 level map and the Sec. 5.1 time-averaged sensor: the average over 10 sensor steps of
    the 8^d tile maxima (block max over tiles), and the affine and fitted level maps of the last and
    the averaged block maxima, against the oracle.  Levels are compared outside a band around the
    integer decision values whose width follows the sensor tolerance (kband relative in K)."""
    tau, every, nsens, b = 0.6, 3, 10, 16
    lat, o = make(L, q, *dims, tau, getattr(L, "LBM_" + dtype))
    L.lbm_set_sensor_every(lat.h, every)
    L.lbm_set_sensor_average(lat.h, 1)
    # a seeded perturbed start gives every block a sensor value well above round-off (the fitted
    # map is defined by the smallest block maximum)
    lat.set_populations(perturbed(o, seed=5 + q, amp=0.01))
    f = lat.populations()
    tile_sum = None
    for _ in range(nsens):
        lat.step(every)
        f, K = o.run(f, every, sensor_last=True)
        t8 = O.block_max(K, 8)
        tile_sum = t8 if tile_sum is None else tile_sum + t8
    # block max over tiles of the averaged tile maxima
    tiles = (tile_sum / nsens).reshape(-(-dims[2] // 8) if q == 19 else 1, -(-dims[1] // 8),
                                       -(-dims[0] // 8))
    ref_avg = O.block_max(tiles, 2)  # 2 x 2 (x 2) tiles per 16-block
    got_avg, n = lat.sensor_average(b)
    assert n == nsens
    assert rel(got_avg, ref_avg) < max(kband, 1e-12)
    ref_last = O.block_max(K, b)
    for src, ref in ((False, ref_last), (True, ref_avg)):
        a_, b_ = 0.75, 9.0
        got = lat.levels(b, a_, b_, 0, 5, average=src)
        keep = O.levels_agree(got, ref, a_, b_, 0.0)
        near = np.array([abs(a_ * np.log2(m) + b_ - round(a_ * np.log2(m) + b_)) < 3 * a_ * kband
                         for m in ref])
        keep &= ~near
        assert np.array_equal(got[keep], O.levels_affine(ref, a_, b_, 0, 5)[keep]), src
        assert keep.sum() > 0.8 * len(ref)
        fit = lat.levels_fit(b, 1, 3, average=src)
        af, bf = O.levels_fit_params(ref, 1, 3)
        near = np.array([abs(af * np.log2(m) + bf - round(af * np.log2(m) + bf)) < 3 * af * kband + 1e-9
                         for m in ref])
        assert np.array_equal(fit[~near], O.levels_fit(ref, 1, 3)[~near]), src
        assert fit.min() == 1 and fit.max() == 3
    lat.close()


# ------------------------------------------------------- 512^3 16-bit storage, full size, sampled
def decode16(raw16, dtype_name):
    """Stored 16-bit deviations f - w_i as float64."""
    if dtype_name == "F16S":
        return raw16.view(np.float16).astype(np.float64)
    return (raw16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("dims,dtype_name,rel_store", [
    ((512, 512, 512), "F16S", 2.0 ** -10), ((512, 512, 512), "BF16S", 2.0 ** -7),
    ((1024, 1024, 208), "F16S", 2.0 ** -10)])
def test_cavity_d3q19_16bit_full_size_sampled(L, dims, dtype_name, rel_store):
    """The 512^3 D3Q19 mixed-precision workloads in the benchmark's launch configuration (the
    two-cell kernel, sensor every step), and a 1024 x 1024 x 208 lattice where 20 x cells exceeds
    2^32, so the automatic choice falls back to the one-cell kernel with 64-bit offsets: one step
    from a seeded perturbed 16-bit state.  The oracle evaluates sampled sub-boxes of 20^3 cells
    taken from the decoded state (corners under the lid, edges, faces, the middle): every cell
    whose pull sources lie in the sub-box, or beyond a face that is a wall of the full lattice, has
    the same inputs as in the full lattice.  Outputs are compared in deviation form within the
    16-bit storage rounding (2^-11 / 2^-8 of the value, with a factor 2 margin, plus 1e-7 absolute
    for values in the half subnormal range), and the block maxima of 16^3 blocks against the
    oracle's within 1e-5 (FP32 arithmetic on identical stored inputs)."""
    nx, ny, nz = dims
    q = 19
    tau = O.tau_from_re(0.1, nx, 1000.0)
    lat = L.Lattice(q, nx, ny, nz, tau, dtype=getattr(L, "LBM_" + dtype_name), lid=(0.1, 0.0))
    L.lbm_set_sensor_every(lat.h, 1)
    c, w, _ = O.lattice(q)
    N = nx * ny * nz
    raw = seeded.stored_deviations16(512 + nz, w, N, 0.03, dtype_name)
    lat.set_raw(raw.view(np.uint8).reshape(-1))
    lat.step(1)
    out = lat.raw().view(np.uint16).reshape(q, nz, ny, nx)
    gmax = lat.sensor(16)
    lat.close()
    raw = raw.reshape(q, nz, ny, nx)
    S = 20
    origins = [(0, 0, 0), (nx - S, ny - S, nz - S), (0, ny - S, 0), (nx - S, ny - S, 0),
               (nx - S, 0, nz - S), (nx // 2, ny // 2, nz // 2), (0, ny // 3, nz - S),
               (nx // 4, ny - S, nz // 2)]
    checked = 0
    for (x0, y0, z0) in origins:
        sub = decode16(raw[:, z0:z0 + S, y0:y0 + S, x0:x0 + S].copy(), dtype_name)
        f_sub = sub + w[:, None, None, None]
        o = O.Oracle(q, S, S, S, tau, lid=(0.1, 0.0, 0.0) if y0 + S == ny else (0.0, 0.0, 0.0))
        ok = []
        for a0, n_ax in ((x0, nx), (y0, ny), (z0, nz)):
            loc = np.arange(S)
            good = (loc >= 1) & (loc <= S - 2)
            good |= (loc == 0) & (a0 == 0)
            good |= (loc == S - 1) & (a0 + S == n_ax)
            ok.append(good)
        zz, yy, xx = np.meshgrid(np.where(ok[2])[0], np.where(ok[1])[0], np.where(ok[0])[0],
                                 indexing="ij")
        cells = ((zz * S + yy) * S + xx).reshape(-1)
        ref, K = o.step_cells(f_sub, cells)
        got = decode16(out[:, z0:z0 + S, y0:y0 + S, x0:x0 + S].copy(), dtype_name).reshape(q, -1)
        got = got[:, cells].T
        dref = ref - w[None, :]
        err = np.abs(got - dref)
        # 1e-7 absolute: the half spacing below 2^-14 is 2^-24, plus FP32 arithmetic
        assert (err <= rel_store * np.abs(dref) + 1e-7).all(), (x0, y0, z0, err.max())
        checked += len(cells)
    assert checked > 30000
    # sampled 16^3 blocks with their one-cell margin (or a real wall) inside an 18^3 sub-box
    nbx, nby, nbz = nx // 16, ny // 16, nz // 16
    for (bx, by, bz) in ((0, 0, 0), (nbx - 1, nby - 1, nbz - 1), (0, nby - 1, nbz - 1),
                         (nbx // 2, nby - 1, 3), (7, 11, 12)):
        x0, y0, z0 = [max(0, min(n_ax - 18, 16 * b - 1))
                      for b, n_ax in ((bx, nx), (by, ny), (bz, nz))]
        sub = decode16(raw[:, z0:z0 + 18, y0:y0 + 18, x0:x0 + 18].copy(), dtype_name)
        o = O.Oracle(q, 18, 18, 18, tau, lid=(0.1, 0.0, 0.0) if y0 + 18 == ny else (0.0, 0.0, 0.0))
        zz, yy, xx = np.meshgrid(np.arange(16) + 16 * bz - z0, np.arange(16) + 16 * by - y0,
                                 np.arange(16) + 16 * bx - x0, indexing="ij")
        _, K = o.step_cells(sub + w[:, None, None, None], ((zz * 18 + yy) * 18 + xx).reshape(-1))
        bidx = (bz * nby + by) * nbx + bx
        assert abs(gmax[bidx] - K.max()) / K.max() < 1e-5, (bx, by, bz)


# ------------------------------------------------- flag calls: block maxima and flags in one launch
@pytest.mark.parametrize("q,dims,dtype,block,state", [
    (19, (48, 40, 32), "F32", 8, "rest"),        # every K is 0: all keys tie
    (19, (48, 40, 32), "F32", 16, "perturbed"),
    (19, (48, 40, 32), "F32", 8, "nan"),         # one NaN population: its block's max is NaN
    (9, (96, 80, 1), "F64", 8, "perturbed"),
    (9, (2048, 1024, 1), "F32", 8, "perturbed"),  # 32768 blocks: the two-launch fallback
])
def test_flag_calls_match_the_flag_builder(L, q, dims, dtype, block, state):
    """lbm_flag / lbm_flag_top form the block maxima from the tile maxima and the flags in one
    launch (one CTA with the keys in shared memory for the top fraction).  On the lattice's own
    block maxima (lbm_sensor_dev) they must equal lbm_flags_from_maxima, the separate flag builder
    that the oracle tests pin bit for bit: both rules, ties (ordered by block index), NaN blocks,
    FP32 and FP64 maxima, and a block count above the one-CTA limit."""
    import torch

    nx, ny, nz = dims
    lid = (0.0, 0.0) if state == "rest" else (0.1, 0.0)  # at rest with a resting lid K = 0
    lat = L.Lattice(q, nx, ny, nz, 0.7, dtype=getattr(L, "LBM_" + dtype), lid=lid)
    if state != "rest":
        c, w, _ = O.lattice(q)
        f = w[:, None, None, None] * (1.0 + seeded.relative_perturbation(
            31 + nx, (q, nz, ny, nx), 0.02))
        if state == "nan":
            f[3, nz // 2, ny // 3, nx // 4] = np.nan
        lat.set_populations(f)
    L.lbm_set_sensor_every(lat.h, 1)
    lat.step(1)
    nb = L.lbm_nblocks(lat.h, block)
    maxima = torch.empty(nb, dtype=torch.float64, device="cuda")
    L.lbm_sensor_dev(lat.h, block, maxima)
    ref = torch.empty(nb, dtype=torch.int8, device="cuda")
    m = maxima.cpu().numpy()
    finite = m[np.isfinite(m)]
    T = float(np.median(finite)) if finite.size else 1.0
    for rule, param, call in ((L.LBM_FLAG_TOP, 0.1, lat.flag_top), (L.LBM_FLAG_TOP, 0.5, lat.flag_top),
                              (L.LBM_FLAG_THRESHOLD, T, lat.flag)):
        got = call(param, block=block)
        L.lbm_flags_from_maxima(maxima, L.LBM_F64, nb, rule, param, ref)
        torch.cuda.synchronize()
        assert np.array_equal(got, ref.cpu().numpy()), (rule, param)
        if rule == L.LBM_FLAG_TOP:
            assert int((got == 1).sum()) == int(np.ceil(param * nb))
    if state == "rest":
        assert (m == 0).all()
        top = lat.flag_top(0.1, block=block)
        assert top[:int(np.ceil(0.1 * nb))].all() and not top[int(np.ceil(0.1 * nb)):].any()
    if state == "nan":
        assert np.isnan(m).sum() == 1 and lat.flag_top(0.1, block=block)[np.isnan(m)].all()
    lat.close()
