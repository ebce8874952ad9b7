"""Failure detection and checkpoint/resume through the C ABI, with failures made on the host side
or by a shortened wait limit (no GPU fault is ever provoked).

* an allocation that fails (lbm_debug_fail_alloc makes the library's k-th next device allocation
  report cudaErrorMemoryAllocation without allocating) gives LBM_ENOMEM, leaks no device memory,
  and the call succeeds when retried, with the same results as an undisturbed handle;
* a bounded wait that runs out (lbm_debug_hold_copies stops the TMA-staged kernels' producers
  from issuing copies, so the consumers wait for something that never comes, and
  lbm_debug_set_wait_limit shortens their limit to 1 ms) makes the next synchronising call return
  LBM_ETIMEOUT; the kernel returns with nothing in flight, so the context stays usable: after
  lbm_reset the handle runs bit for bit like a fresh one;
* a checkpoint file written by lbm_checkpoint_save resumes the run bit for bit; a corrupted,
  truncated or foreign file is refused.
"""
import os

import numpy as np
import pytest

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


def free_bytes():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def populations_after(L, steps, dims=(96, 96, 96)):
    h = L.lbm_create(L.LBM_D3Q19, *dims, 0.6)
    try:
        L.lbm_step(h, steps)
        out = np.empty(19 * int(np.prod(dims)))
        L.lbm_get_populations(h, out)
        return out
    finally:
        L.lbm_destroy(h)


def test_allocation_failure_reports_enomem_and_leaks_nothing(L):
    dims = (96, 96, 96)  # 2 x 67 MB of populations: a leak would show in the free memory
    ref = populations_after(L, 3, dims)
    free0 = free_bytes()
    failed = 0
    for k in range(12):
        h = L.lbm_create(L.LBM_D3Q19, *dims, 0.6)
        try:
            L.lbm_debug_fail_alloc(k)
            try:
                L.lbm_step(h, 1)
                steps = 1
            except L.LbmError as e:
                assert e.status == L.LBM_ENOMEM, e
                assert "cudaMalloc" in L.lbm_last_message()
                failed += 1
                steps = 0
            L.lbm_debug_fail_alloc(-1)
            L.lbm_step(h, 3 - steps)  # the retry completes the allocations
            out = np.empty(19 * int(np.prod(dims)))
            L.lbm_get_populations(h, out)
            assert np.array_equal(out, ref), k
        finally:
            L.lbm_debug_fail_alloc(-1)
            L.lbm_destroy(h)
    # a step allocates the sensor scratch (7 buffers) and the two population buffers: each of
    # those 9 allocations was made to fail once
    assert failed == 9
    assert abs(free_bytes() - free0) < 8 << 20


def test_network_allocation_failure(L):
    free0 = free_bytes()
    for k in range(7):  # parameters, gradients, two moments, BF16 copy, loss partials, loss
        L.lbm_debug_fail_alloc(k)
        with pytest.raises(L.LbmError) as ei:
            L.lbm_net_create(3, 16)
        assert ei.value.status == L.LBM_ENOMEM
    L.lbm_debug_fail_alloc(-1)
    n = L.lbm_net_create(3, 16)
    L.lbm_net_destroy(n)
    assert abs(free_bytes() - free0) < 8 << 20


@pytest.mark.parametrize("variant,dtype", [("TMA", "F32"), ("TMA_PAIR", "F16S")])
def test_bounded_wait_runs_out_and_the_context_survives(L, variant, dtype):
    dims = (64, 64, 64)
    dt = getattr(L, "LBM_" + dtype)
    kv = getattr(L, "LBM_KERNEL_" + variant)
    lat = L.Lattice(L.LBM_D3Q19, *dims, 0.6, dtype=dt, lid=(0.1, 0.0))
    L.lbm_set_kernel_variant(lat.h, kv)
    # the producers issue nothing: the consumers' first wait runs out after 1 ms
    L.lbm_debug_hold_copies(lat.h, 1)
    L.lbm_debug_set_wait_limit(lat.h, 1_000_000)
    L.lbm_step(lat.h, 2)
    with pytest.raises(L.LbmError) as ei:
        lat.sensor(16)  # synchronises and reads the kernels' error word
    assert ei.value.status == L.LBM_ETIMEOUT
    # the default again; lbm_reset clears the error and restarts from rest
    L.lbm_debug_hold_copies(lat.h, 0)
    L.lbm_debug_set_wait_limit(lat.h, 0)
    L.lbm_reset(lat.h)
    L.lbm_step(lat.h, 10)
    got = lat.populations()
    k_got = lat.sensor(16)
    lat.close()
    fresh = L.Lattice(L.LBM_D3Q19, *dims, 0.6, dtype=dt, lid=(0.1, 0.0))
    L.lbm_set_kernel_variant(fresh.h, kv)
    L.lbm_step(fresh.h, 10)
    assert np.array_equal(got, fresh.populations())
    assert np.array_equal(k_got, fresh.sensor(16))
    fresh.close()


@pytest.mark.parametrize("dtype", ["F32", "F16S"])
def test_checkpoint_file_resumes_bit_for_bit(L, dtype, tmp_path):
    dims = (40, 36, 33)
    dt = getattr(L, "LBM_" + dtype)
    a = L.Lattice(L.LBM_D3Q19, *dims, 0.57, dtype=dt, lid=(0.08, 0.02))
    L.lbm_set_periodic(a.h, L.LBM_PERIODIC_Z)
    L.lbm_step(a.h, 30)
    path = str(tmp_path / "cavity.ckpt")
    L.lbm_checkpoint_save(a.h, path)
    assert os.path.getsize(path) == 88 + L.lbm_population_bytes(a.h)
    L.lbm_step(a.h, 20)
    ref = a.raw()
    # a handle with other parameters takes the file's tau, lid, periodic mask and step counter
    b = L.Lattice(L.LBM_D3Q19, *dims, 0.9, dtype=dt, lid=(0.0, 0.0))
    L.lbm_checkpoint_load(b.h, path)
    assert L.lbm_steps_done(b.h) == 30
    L.lbm_step(b.h, 20)
    assert np.array_equal(b.raw(), ref)
    assert L.lbm_steps_done(b.h) == 50
    # refused files
    blob = open(path, "rb").read()
    bad = bytearray(blob)
    bad[88 + 1234] ^= 0x40
    open(path, "wb").write(bytes(bad))
    with pytest.raises(L.LbmError) as ei:
        L.lbm_checkpoint_load(b.h, path)
    assert ei.value.status == L.LBM_EIO
    open(path, "wb").write(blob[:-100])
    with pytest.raises(L.LbmError) as ei:
        L.lbm_checkpoint_load(b.h, path)
    assert ei.value.status == L.LBM_EIO
    open(path, "wb").write(b"not a checkpoint" * 10)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_checkpoint_load(b.h, path)
    assert ei.value.status == L.LBM_EIO
    open(path, "wb").write(blob)
    c = L.Lattice(L.LBM_D3Q19, 40, 36, 32, 0.57, dtype=dt)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_checkpoint_load(c.h, path)
    assert ei.value.status == L.LBM_EINVAL
    for lat in (a, b, c):
        lat.close()
