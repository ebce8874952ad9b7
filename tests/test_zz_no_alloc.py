"""lbm_step_noalloc: the entry point for callers that may not allocate device memory.

Such callers (applications that serve all device memory from their own pool, or latency-critical
loops that cannot pay for a cudaMalloc after set-up) call it with buffers they already own; the
library keeps its scratch in a fixed device array.  This file checks, through the C ABI, that two
calls in a row give the same populations and block maxima as the handle-based path (lbm_step +
lbm_sensor), and that a lattice beyond the scratch limit is refused.  It is named to be collected
last; it also passes on its own in a fresh process (its first call then does the per-device
set-up).
"""
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


@pytest.mark.parametrize("q,dims,dtype,block", [
    (19, (40, 36, 33), "F32", 16),
    (9, (70, 45, 1), "F64", 8),
    (19, (24, 16, 20), "BF16S", 8),
    (19, (256, 256, 256), "F32", 16),  # the benchmark lattice (one-cell FP32 kernel)
    (9, (512, 384, 1), "F32", 16),  # FP32 D2Q9 above 2^17 cells: the two-cell kernel
])
def test_noalloc_matches_handle_path_two_calls(L, q, dims, dtype, block):
    import torch

    nx, ny, nz = dims
    tau, lid = 0.62, (0.1, 0.02 if q == 19 else 0.0)
    dt = getattr(L, "LBM_" + dtype)
    o = O.Oracle(q, nx, ny, nz, tau)
    f0 = o.w[:, None, None, None] * (1.0 + seeded.relative_perturbation(5, o.shape, 0.02))

    # handle path: the existing entry points
    lat = L.Lattice(q, nx, ny, nz, tau, dtype=dt, lid=lid)
    lat.set_populations(f0)
    raw0 = lat.raw()
    L.lbm_set_sensor_every(lat.h, 1)
    ref = []
    for _ in range(2):
        lat.step(1)
        ref.append((lat.raw(), lat.sensor(block)))
    lat.close()

    # no-allocation path on caller-owned buffers, starting from the same stored bytes
    nbytes = raw0.nbytes
    a = torch.from_numpy(raw0.copy()).cuda()
    b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    nb = (-(-nx // block)) * (-(-ny // block)) * (-(-nz // block) if q == 19 else 1)
    maxima = torch.empty(nb, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    src, dst = a, b
    for k in range(2):
        maxima.fill_(-1.0)
        L.lbm_step_noalloc(q, dt, nx, ny, nz, tau, lid[0], lid[1], 0, src, dst, block, maxima,
                           stream)
        torch.cuda.synchronize()
        got_f = dst.cpu().numpy()
        got_m = maxima.cpu().numpy()
        ref_f, ref_m = ref[k]
        # same kernels on the same bytes: identical results (tolerance 0 within the FP32/FP64
        # tolerances the other tests use)
        assert np.array_equal(got_f, ref_f), k
        assert np.array_equal(got_m, ref_m), k
        src, dst = dst, src


def test_noalloc_rejects_lattices_beyond_the_limit(L):
    import torch

    buf = torch.empty(16, dtype=torch.float32, device="cuda")
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LbmError) as ei:
        # 1024^3 needs 128^3 tiles > LBM_NOALLOC_MAX_TILES; refused before any device work
        L.lbm_step_noalloc(L.LBM_D3Q19, L.LBM_F32, 1024, 1024, 1024, 0.6, 0.1, 0.0, 0, buf,
                           out, 16, out, None)
    assert ei.value.status == L.LBM_EINVAL
    assert "LBM_NOALLOC_MAX_TILES" in L.lbm_last_message()
    assert L.LBM_NOALLOC_MAX_TILES == 262144
