"""The C-ABI library builds, loads and exports every symbol include/lbm.h declares; argument
validation works without a GPU (no compute calls are made here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1507_06767_gb300 as pkg

    return pkg


def test_every_declared_symbol_is_exported(L):
    names = L.exported_symbols()
    assert len(names) >= 35
    lib = ctypes.CDLL(L.lbm.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    nm = subprocess.run(["nm", "-D", "--defined-only", L.lbm.LIB_PATH], capture_output=True,
                        text=True, check=True).stdout
    exported = set(re.findall(r"\b[TW]\s+(lbm_\w+)", nm))
    assert set(names) == exported, set(names) ^ exported
    # and the Python binding exposes each under the same name
    for n in names:
        assert callable(getattr(L, n)), n


def test_header_constants(L):
    assert (L.LBM_D2Q9, L.LBM_D3Q19) == (9, 19)
    assert (L.LBM_F64, L.LBM_F32, L.LBM_F16S, L.LBM_BF16S) == (0, 1, 2, 3)
    assert L.LBM_OK == 0 and L.LBM_EINVAL == -1 and L.LBM_ENOTSUP == -6
    assert L.LBM_TILE == 8
    assert L.lbm_version() == 100
    assert L.lbm_strerror(L.LBM_ENUMERIC) == "non-finite populations"


@pytest.mark.parametrize("args", [(7, 8, 8, 1, 0.8), (9, 8, 8, 2, 0.8), (19, 0, 8, 8, 0.8),
                                  (19, 8, 8, 8, 0.5), (19, 8, 8, 8, float("nan")),
                                  (19, 2048, 2048, 1024, 0.8)])
def test_create_rejects_bad_arguments(L, args):
    with pytest.raises(L.LbmError) as ei:
        L.lbm_create(*args)
    assert ei.value.status == L.LBM_EINVAL
    assert L.lbm_last_error() == L.LBM_EINVAL


def test_host_side_setters_and_queries(L):
    h = L.lbm_create(L.LBM_D3Q19, 40, 36, 33, 0.6)
    try:
        assert L.lbm_population_bytes(h) == 19 * 40 * 36 * 33 * 4
        L.lbm_set_dtype(h, L.LBM_BF16S)
        assert L.lbm_population_bytes(h) == 19 * 40 * 36 * 33 * 2
        assert L.lbm_nblocks(h, 16) == 3 * 3 * 3
        assert L.lbm_nblocks(h, 8) == 5 * 5 * 5
        assert L.lbm_nblocks(h, 12) == 0
        assert L.lbm_steps_done(h) == 0
        for call, args in [(L.lbm_set_dtype, (9,)), (L.lbm_set_block, (12,)),
                           (L.lbm_set_tau, (0.4,)), (L.lbm_set_periodic, (8,)),
                           (L.lbm_set_sensor_every, (-1,)), (L.lbm_step, (-2,)),
                           (L.lbm_set_lid, (float("inf"), 0.0))]:
            with pytest.raises(L.LbmError) as ei:
                call(h, *args)
            assert ei.value.status == L.LBM_EINVAL, call
        with pytest.raises(L.LbmError) as ei:
            L.lbm_blocks_step(h)  # NULL batch
        assert ei.value.status == L.LBM_EINVAL
        leaf = np.zeros(1, dtype=np.int8)
        batch = L.LevelBatch(1, 1, 1, 40, 0, leaf.ctypes.data, 0, None)
        with pytest.raises(L.LbmError) as ei:  # BF16 storage (set above) is not supported
            L.lbm_blocks_step(h, batch)
        assert ei.value.status == L.LBM_ENOTSUP
        L.lbm_set_block(h, 32)
        L.lbm_set_lid(h, 0.05, 0.01)
        L.lbm_set_sensor_every(h, 10)
    finally:
        L.lbm_destroy(h)


def test_flags_from_maxima_validation(L):
    for args in [(0, L.LBM_F16S, 4, L.LBM_FLAG_TOP, 0.1, 0), (0, L.LBM_F32, -1, 0, 0.1, 0),
                 (0, L.LBM_F32, 4, L.LBM_FLAG_TOP, 1.5, 0), (0, L.LBM_F32, 4, 7, 0.1, 0)]:
        with pytest.raises(L.LbmError) as ei:
            L.lbm_flags_from_maxima(*args)
        assert ei.value.status == L.LBM_EINVAL
    # n == 0 is a no-op
    L.lbm_flags_from_maxima(0, L.LBM_F32, 0, L.LBM_FLAG_TOP, 0.1, 0)


def test_product_does_not_reach_the_oracle():
    """The product package never imports, links or loads anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1507_06767_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in src.lower(), fn
    nm = subprocess.run(["nm", "-D", os.path.join(pkg, "_build", "liblbm.so")],
                        capture_output=True, text=True).stdout
    assert "orc_" not in nm
