"""Python binding of the C ABI in include/lbm.h (ctypes; argument marshalling only).

Every function of the C ABI is exposed under the same name and raises ``LbmError`` on a negative
status.  Device memory for the two population buffers can come from PyTorch (``Lattice`` does that
with ``lbm_attach``); streams are passed as raw ``cudaStream_t`` handles, e.g.
``torch.cuda.current_stream().cuda_stream``.  Nothing here computes any part of the method: the
library runs every step in its CUDA kernels, and importing this module fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lbm.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)


def _header_constants():
    out = {}
    with open(HEADER) as fh:
        for m in re.finditer(r"#define\s+(LBM_\w+)\s+\(?(-?\d+)\)?", fh.read()):
            out[m.group(1)] = int(m.group(2))
    return out


globals().update(_header_constants())

_h = ctypes.c_void_p
_i, _d, _sz, _ll = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_longlong
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i8p = ctypes.c_void_p

_SIGS = {
    "lbm_last_error": (_i, []),
    "lbm_last_message": (ctypes.c_char_p, []),
    "lbm_strerror": (ctypes.c_char_p, [_i]),
    "lbm_version": (_i, []),
    "lbm_create": (_h, [_i, _i, _i, _i, _d]),
    "lbm_destroy": (_i, [_h]),
    "lbm_set_dtype": (_i, [_h, _i]),
    "lbm_set_lid": (_i, [_h, _d, _d]),
    "lbm_set_periodic": (_i, [_h, _i]),
    "lbm_set_tau": (_i, [_h, _d]),
    "lbm_set_stream": (_i, [_h, _vp]),
    "lbm_set_sensor_every": (_i, [_h, _i]),
    "lbm_set_sensor_field": (_i, [_h, _i]),
    "lbm_set_block": (_i, [_h, _i]),
    "lbm_set_profiling": (_i, [_h, _i]),
    "lbm_set_graphs": (_i, [_h, _i]),
    "lbm_set_kernel_variant": (_i, [_h, _i]),
    "lbm_attach": (_i, [_h, _vp, _vp, _sz]),
    "lbm_population_bytes": (_sz, [_h]),
    "lbm_nblocks": (_i, [_h, _i]),
    "lbm_steps_done": (_ll, [_h]),
    "lbm_reset": (_i, [_h]),
    "lbm_step": (_i, [_h, _i]),
    "lbm_sensor": (_i, [_h, _i, _vp]),
    "lbm_sensor_dev": (_i, [_h, _i, _vp]),
    "lbm_flag": (_i, [_h, _d, _vp]),
    "lbm_flag_dev": (_i, [_h, _d, _vp]),
    "lbm_flag_top": (_i, [_h, _d, _vp]),
    "lbm_flag_top_dev": (_i, [_h, _d, _vp]),
    "lbm_flags_from_maxima": (_i, [_vp, _i, _i, _i, _d, _vp, _vp]),
    "lbm_get_populations": (_i, [_h, _vp]),
    "lbm_set_populations": (_i, [_h, _vp]),
    "lbm_get_raw": (_i, [_h, _vp, _sz]),
    "lbm_set_raw": (_i, [_h, _vp, _sz]),
    "lbm_get_moments": (_i, [_h, _vp, _vp]),
    "lbm_get_sensor_field": (_i, [_h, _vp]),
    "lbm_conservation": (_i, [_h, _dp, _dp]),
    "lbm_kernel_time": (_i, [_h, _dp, ctypes.POINTER(_ll)]),
    "lbm_blocks_step": (_i, [_h, _vp]),
    "lbm_blocks_get": (_i, [_h, _i, _i, _vp]),
    "lbm_blocks_set": (_i, [_h, _i, _i, _vp]),
    "lbm_blocks_info": (_i, [_h, _i, ctypes.POINTER(_i), _dp, ctypes.POINTER(_i),
                             ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_ll)]),
    "lbm_set_sensor_average": (_i, [_h, _i]),
    "lbm_sensor_average": (_i, [_h, _i, _vp, ctypes.POINTER(_ll)]),
    "lbm_levels": (_i, [_h, _i, _d, _d, _i, _i, _i, _vp]),
    "lbm_levels_fit": (_i, [_h, _i, _i, _i, _i, _vp]),
    "lbm_step_noalloc": (_i, [_i, _i, _i, _i, _i, _d, _d, _d, _i, _vp, _vp, _i, _vp, _vp]),
    "lbm_regrid": (_i, [_h, _vp, _vp, _vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_ll), _vp]),
    "lbm_block_features": (_i, [_h, _i, _vp]),
    "lbm_blocks_set_fusion": (_i, [_h, _i]),
    "lbm_blocks_set_step_form": (_i, [_h, _i]),
    "lbm_blocks_set_schedule": (_i, [_h, _i]),
    "lbm_blocks_cycle_form": (_i, [_h]),
    "lbm_blocks_schedule": (_i, [_h, _i, ctypes.POINTER(_i), ctypes.POINTER(_i),
                                 ctypes.POINTER(_i)]),
    "lbm_net_create": (_vp, [_i, _i]),
    "lbm_net_destroy": (None, [_vp]),
    "lbm_net_set_stream": (_i, [_vp, _vp]),
    "lbm_net_param_count": (_i, [_vp]),
    "lbm_net_set_normalisation": (_i, [_vp, _vp, _vp]),
    "lbm_net_set_params": (_i, [_vp, _vp]),
    "lbm_net_get_params": (_i, [_vp, _vp]),
    "lbm_net_get_grads": (_i, [_vp, _vp]),
    "lbm_net_set_grads": (_i, [_vp, _vp]),
    "lbm_net_forward": (_i, [_vp, _vp, _i, _i, _i, _vp]),
    "lbm_net_backward": (_i, [_vp, _vp, _vp, _i, _i, _i, _dp]),
    "lbm_net_adam": (_i, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "lbm_net_train_step": (_i, [_vp, _vp, _vp, _i, _i, _i, ctypes.c_float, _dp]),
    "lbm_net_log_targets": (_i, [_vp, _ll, ctypes.c_float, ctypes.c_float, _vp, _vp]),
    "lbm_net_to_maxima": (_i, [_vp, _ll, ctypes.c_float, _vp, _vp]),
    "lbm_net_log_residual": (_i, [_vp, _vp, _ll, ctypes.c_float, _vp, _vp]),
    "lbm_net_to_maxima_residual": (_i, [_vp, _vp, _ll, ctypes.c_float, _vp, _vp]),
    "lbm_net_get_buffer": (_i, [_vp, _i, _vp, _sz]),
    "lbm_flags_agreement": (_i, [_vp, _vp, _i, _vp, _vp]),
    "lbm_flags_judge_select": (_i, [_vp, _vp, _vp, _i, _d, _vp, _vp, _vp, _vp]),
    "lbm_gather_rows": (_i, [_vp, _ll, _sz, _vp, _i, _vp, _vp, _vp]),
    "lbm_checkpoint_save": (_i, [_h, ctypes.c_char_p]),
    "lbm_checkpoint_load": (_i, [_h, ctypes.c_char_p]),
    "lbm_debug_fail_alloc": (_i, [_i]),
    "lbm_debug_set_wait_limit": (_i, [_h, _ll]),
    "lbm_debug_hold_copies": (_i, [_h, _i]),
    "lbm_set_halo": (_i, [_h, _i]),
    "lbm_halo_size": (_i, [_h, ctypes.POINTER(_ll), ctypes.POINTER(_ll)]),
    "lbm_halo_export": (_i, [_h, _i, _vp, _i]),
    "lbm_halo_import": (_i, [_h, _i, _vp, _i]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.lbm_last_message().decode(errors="replace")
        name = _lib.lbm_strerror(status).decode()
        super().__init__(f"{where}: {name} ({status}): {msg}")


def _ck(status: int, where: str) -> int:
    if status < 0:
        raise LbmError(status, where)
    return status


def _ptr(a):
    """Address of a numpy array, a torch tensor, or an int address."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(f"cannot take the address of {type(a)}")


# ----------------------------------------------------------------------------- C-ABI functions
def lbm_last_error() -> int:
    return _lib.lbm_last_error()


def lbm_last_message() -> str:
    return _lib.lbm_last_message().decode(errors="replace")


def lbm_strerror(status: int) -> str:
    return _lib.lbm_strerror(status).decode()


def lbm_version() -> int:
    return _lib.lbm_version()


def lbm_create(lattice: int, nx: int, ny: int, nz: int, tau: float) -> int:
    h = _lib.lbm_create(lattice, nx, ny, nz, tau)
    if not h:
        raise LbmError(_lib.lbm_last_error(), "lbm_create")
    return h


def _wrap(name, *conv):
    f = getattr(_lib, name)

    def call(*args):
        return _ck(f(*args), name)

    call.__name__ = name
    return call


lbm_destroy = _wrap("lbm_destroy")
lbm_set_dtype = _wrap("lbm_set_dtype")
lbm_set_lid = _wrap("lbm_set_lid")
lbm_set_periodic = _wrap("lbm_set_periodic")
lbm_set_tau = _wrap("lbm_set_tau")
lbm_set_sensor_every = _wrap("lbm_set_sensor_every")
lbm_set_sensor_field = _wrap("lbm_set_sensor_field")
lbm_set_block = _wrap("lbm_set_block")
lbm_set_profiling = _wrap("lbm_set_profiling")
lbm_set_graphs = _wrap("lbm_set_graphs")
lbm_set_kernel_variant = _wrap("lbm_set_kernel_variant")
lbm_reset = _wrap("lbm_reset")
lbm_step = _wrap("lbm_step")
lbm_debug_fail_alloc = _wrap("lbm_debug_fail_alloc")
lbm_debug_set_wait_limit = _wrap("lbm_debug_set_wait_limit")
lbm_debug_hold_copies = _wrap("lbm_debug_hold_copies")


lbm_set_halo = _wrap("lbm_set_halo")


def lbm_halo_size(h):
    """(elements, bytes) of one halo message."""
    n, b = ctypes.c_longlong(), ctypes.c_longlong()
    _ck(_lib.lbm_halo_size(h, ctypes.byref(n), ctypes.byref(b)), "lbm_halo_size")
    return n.value, b.value


def _on_device(a) -> int:
    return int(bool(getattr(a, "is_cuda", False)))


def lbm_halo_export(h, face: int, out) -> int:
    """Writes the populations leaving through `face` into `out` (a numpy array or a host tensor:
    synchronous; a CUDA tensor: asynchronous on the handle's stream)."""
    return _ck(_lib.lbm_halo_export(h, face, _ptr(out), _on_device(out)), "lbm_halo_export")


def lbm_halo_import(h, face: int, arr) -> int:
    """Sets the halo of `face` from `arr` (host memory: synchronous; a CUDA tensor: asynchronous)."""
    return _ck(_lib.lbm_halo_import(h, face, _ptr(arr), _on_device(arr)), "lbm_halo_import")


def lbm_checkpoint_save(h, path) -> int:
    return _ck(_lib.lbm_checkpoint_save(h, os.fsencode(path)), "lbm_checkpoint_save")


def lbm_checkpoint_load(h, path) -> int:
    return _ck(_lib.lbm_checkpoint_load(h, os.fsencode(path)), "lbm_checkpoint_load")


def lbm_set_stream(h, stream) -> int:
    return _ck(_lib.lbm_set_stream(h, stream if stream is None or isinstance(stream, int)
                                   else stream.cuda_stream), "lbm_set_stream")


def lbm_attach(h, a, b, nbytes: int) -> int:
    return _ck(_lib.lbm_attach(h, _ptr(a), _ptr(b), nbytes), "lbm_attach")


def lbm_population_bytes(h) -> int:
    return _lib.lbm_population_bytes(h)


def lbm_nblocks(h, block: int) -> int:
    return _lib.lbm_nblocks(h, block)


def lbm_steps_done(h) -> int:
    return _lib.lbm_steps_done(h)


def lbm_sensor(h, block: int, out) -> int:
    return _ck(_lib.lbm_sensor(h, block, _ptr(out)), "lbm_sensor")


def lbm_sensor_dev(h, block: int, out_dev) -> int:
    return _ck(_lib.lbm_sensor_dev(h, block, _ptr(out_dev)), "lbm_sensor_dev")


def lbm_flag(h, threshold: float, out) -> int:
    return _ck(_lib.lbm_flag(h, threshold, _ptr(out)), "lbm_flag")


def lbm_flag_dev(h, threshold: float, out_dev) -> int:
    return _ck(_lib.lbm_flag_dev(h, threshold, _ptr(out_dev)), "lbm_flag_dev")


def lbm_flag_top(h, frac: float, out) -> int:
    return _ck(_lib.lbm_flag_top(h, frac, _ptr(out)), "lbm_flag_top")


def lbm_flag_top_dev(h, frac: float, out_dev) -> int:
    return _ck(_lib.lbm_flag_top_dev(h, frac, _ptr(out_dev)), "lbm_flag_top_dev")


def lbm_flags_from_maxima(maxima_dev, maxima_dtype: int, n: int, rule: int, param: float, out_dev,
                          stream=None) -> int:
    s = stream if stream is None or isinstance(stream, int) else stream.cuda_stream
    return _ck(_lib.lbm_flags_from_maxima(_ptr(maxima_dev), maxima_dtype, n, rule, param,
                                          _ptr(out_dev), s), "lbm_flags_from_maxima")


lbm_set_sensor_average = _wrap("lbm_set_sensor_average")


def lbm_sensor_average(h, block: int, out):
    """Writes the time-averaged block maxima into out; returns the number of averaged steps."""
    n = ctypes.c_longlong()
    _ck(_lib.lbm_sensor_average(h, block, _ptr(out), ctypes.byref(n)), "lbm_sensor_average")
    return n.value


def lbm_levels(h, block: int, a: float, b: float, lmin: int, lmax: int, source: int, out) -> int:
    return _ck(_lib.lbm_levels(h, block, a, b, lmin, lmax, source, _ptr(out)), "lbm_levels")


def lbm_levels_fit(h, block: int, lmin: int, lmax: int, source: int, out) -> int:
    return _ck(_lib.lbm_levels_fit(h, block, lmin, lmax, source, _ptr(out)), "lbm_levels_fit")


def lbm_get_populations(h, out) -> int:
    return _ck(_lib.lbm_get_populations(h, _ptr(out)), "lbm_get_populations")


def lbm_set_populations(h, arr) -> int:
    return _ck(_lib.lbm_set_populations(h, _ptr(arr)), "lbm_set_populations")


def lbm_get_raw(h, out, nbytes: int) -> int:
    return _ck(_lib.lbm_get_raw(h, _ptr(out), nbytes), "lbm_get_raw")


def lbm_set_raw(h, arr, nbytes: int) -> int:
    return _ck(_lib.lbm_set_raw(h, _ptr(arr), nbytes), "lbm_set_raw")


def lbm_get_moments(h, rho, u) -> int:
    return _ck(_lib.lbm_get_moments(h, _ptr(rho), _ptr(u)), "lbm_get_moments")


def lbm_get_sensor_field(h, out) -> int:
    return _ck(_lib.lbm_get_sensor_field(h, _ptr(out)), "lbm_get_sensor_field")


def lbm_conservation(h):
    """Returns (mass, momentum[3]); raises LbmError(LBM_ENUMERIC) on non-finite populations."""
    m = ctypes.c_double()
    j = (ctypes.c_double * 3)()
    _ck(_lib.lbm_conservation(h, ctypes.byref(m), j), "lbm_conservation")
    return m.value, np.array(list(j))


def lbm_kernel_time(h):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _ck(_lib.lbm_kernel_time(h, ctypes.byref(ms), ctypes.byref(n)), "lbm_kernel_time")
    return ms.value, n.value


class LevelBatch(ctypes.Structure):
    """struct lbm_level_batch of include/lbm.h."""
    _fields_ = [("nbx", _i), ("nby", _i), ("nbz", _i), ("edge", _i), ("lmax", _i),
                ("leaf", ctypes.c_void_p), ("cycles", _i), ("block_max", ctypes.c_void_p)]


def lbm_blocks_step(h, batch=None) -> int:
    p = ctypes.byref(batch) if isinstance(batch, LevelBatch) else _ptr(batch)
    return _ck(_lib.lbm_blocks_step(h, p), "lbm_blocks_step")


def lbm_blocks_get(h, level: int, block: int, out) -> int:
    return _ck(_lib.lbm_blocks_get(h, level, block, _ptr(out)), "lbm_blocks_get")


def lbm_blocks_set(h, level: int, block: int, arr) -> int:
    return _ck(_lib.lbm_blocks_set(h, level, block, _ptr(arr)), "lbm_blocks_set")


def lbm_blocks_info(h, level: int):
    """(cells per block edge, tau, blocks at the level, threads, cells per thread, cell updates
    per cycle)."""
    n, nb, th, cpt = _i(), _i(), _i(), _i()
    tau = ctypes.c_double()
    cu = ctypes.c_longlong()
    _ck(_lib.lbm_blocks_info(h, level, ctypes.byref(n), ctypes.byref(tau), ctypes.byref(nb),
                             ctypes.byref(th), ctypes.byref(cpt), ctypes.byref(cu)),
        "lbm_blocks_info")
    return n.value, tau.value, nb.value, th.value, cpt.value, cu.value


def lbm_blocks_set_fusion(h, mode: int) -> int:
    return _ck(_lib.lbm_blocks_set_fusion(h, int(mode)), "lbm_blocks_set_fusion")


def lbm_blocks_set_step_form(h, form: int) -> int:
    return _ck(_lib.lbm_blocks_set_step_form(h, int(form)), "lbm_blocks_set_step_form")


def lbm_blocks_set_schedule(h, mode: int) -> int:
    return _ck(_lib.lbm_blocks_set_schedule(h, int(mode)), "lbm_blocks_set_schedule")


def lbm_blocks_cycle_form(h) -> int:
    return _ck(_lib.lbm_blocks_cycle_form(h), "lbm_blocks_cycle_form")


def lbm_blocks_schedule(h, level: int):
    """(form, planes, fused planes) of a level's step schedule; form 0 flat, 1 tiled, 2 flat with
    the address-select gather, 3 two cells per thread."""
    t, p, f = _i(), _i(), _i()
    _ck(_lib.lbm_blocks_schedule(h, int(level), ctypes.byref(t), ctypes.byref(p), ctypes.byref(f)),
        "lbm_blocks_schedule")
    return t.value, p.value, f.value


class RegridParams(ctypes.Structure):
    """struct lbm_regrid_params of include/lbm.h."""
    _fields_ = [("coarsen", _i), ("threshold", _d), ("buffer", _i), ("allowed", ctypes.c_void_p),
                ("nest", _i), ("efficiency", _d), ("min_width", _i)]


class Box(ctypes.Structure):
    """struct lbm_box of include/lbm.h."""
    _fields_ = [("lo", _i * 3), ("hi", _i * 3)]


def lbm_regrid(h, field_dev, params, boxes, max_boxes: int, tags_out=None):
    """Returns (number of boxes, tagged tag cells).  `boxes` is a ctypes array of Box (or an
    address), `field_dev` a device array of doubles or None for the handle's sensor field."""
    nb = _i()
    nt = ctypes.c_longlong()
    bp = boxes if isinstance(boxes, ctypes.Array) else _ptr(boxes)
    st = _lib.lbm_regrid(h, _ptr(field_dev), ctypes.byref(params), bp, int(max_boxes),
                         ctypes.byref(nb), ctypes.byref(nt), _ptr(tags_out))
    _ck(st, "lbm_regrid")
    return nb.value, nt.value


def lbm_block_features(h, block: int, out_dev) -> int:
    return _ck(_lib.lbm_block_features(h, int(block), _ptr(out_dev)), "lbm_block_features")


def lbm_net_log_targets(kmax_dev, n: int, offset: float, floor_k: float, t_dev, stream=None):
    return _ck(_lib.lbm_net_log_targets(_ptr(kmax_dev), int(n), float(offset), float(floor_k),
                                        _ptr(t_dev), stream), "lbm_net_log_targets")


def lbm_net_to_maxima(y_dev, n: int, offset: float, kmax_dev, stream=None):
    return _ck(_lib.lbm_net_to_maxima(_ptr(y_dev), int(n), float(offset), _ptr(kmax_dev), stream),
               "lbm_net_to_maxima")


def lbm_net_log_residual(kmax_next_dev, kmax_now_dev, n: int, floor_k: float, t_dev, stream=None):
    return _ck(_lib.lbm_net_log_residual(_ptr(kmax_next_dev), _ptr(kmax_now_dev), int(n),
                                         float(floor_k), _ptr(t_dev), stream),
               "lbm_net_log_residual")


def lbm_net_to_maxima_residual(y_dev, kmax_now_dev, n: int, floor_k: float, kmax_dev, stream=None):
    return _ck(_lib.lbm_net_to_maxima_residual(_ptr(y_dev), _ptr(kmax_now_dev), int(n),
                                               float(floor_k), _ptr(kmax_dev), stream),
               "lbm_net_to_maxima_residual")


def lbm_net_create(cin: int, hidden: int):
    n = _lib.lbm_net_create(int(cin), int(hidden))
    if not n:
        raise LbmError(_lib.lbm_last_error(), "lbm_net_create")
    return n


def lbm_net_destroy(n) -> None:
    _lib.lbm_net_destroy(n)


def lbm_net_set_stream(n, stream) -> int:
    return _ck(_lib.lbm_net_set_stream(n, stream), "lbm_net_set_stream")


def lbm_net_param_count(n) -> int:
    return _ck(_lib.lbm_net_param_count(n), "lbm_net_param_count")


def lbm_net_set_normalisation(n, shift, scale) -> int:
    return _ck(_lib.lbm_net_set_normalisation(n, _ptr(shift), _ptr(scale)),
               "lbm_net_set_normalisation")


def lbm_net_set_params(n, host) -> int:
    return _ck(_lib.lbm_net_set_params(n, _ptr(host)), "lbm_net_set_params")


def lbm_net_get_params(n, host) -> int:
    return _ck(_lib.lbm_net_get_params(n, _ptr(host)), "lbm_net_get_params")


def lbm_net_get_grads(n, host) -> int:
    return _ck(_lib.lbm_net_get_grads(n, _ptr(host)), "lbm_net_get_grads")


def _stream_handle(stream):
    if stream is None:
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def lbm_flags_agreement(a_dev, b_dev, n: int, out_dev, stream=None) -> int:
    return _ck(_lib.lbm_flags_agreement(_ptr(a_dev), _ptr(b_dev), int(n), _ptr(out_dev),
                                        _stream_handle(stream)), "lbm_flags_agreement")


def lbm_flags_judge_select(pred_prev_dev, exact_now_dev, pred_next_dev, n: int,
                           min_agreement: float, used_dev, agreement_dev=None, fell_back_dev=None,
                           stream=None) -> int:
    return _ck(_lib.lbm_flags_judge_select(_ptr(pred_prev_dev), _ptr(exact_now_dev),
                                           _ptr(pred_next_dev), int(n), float(min_agreement),
                                           _ptr(used_dev), _ptr(agreement_dev),
                                           _ptr(fell_back_dev), _stream_handle(stream)),
               "lbm_flags_judge_select")


def lbm_gather_rows(src_dev, nrows: int, row_bytes: int, idx_dev, count: int, dst_dev, bad_dev,
                    stream=None) -> int:
    return _ck(_lib.lbm_gather_rows(_ptr(src_dev), int(nrows), int(row_bytes), _ptr(idx_dev),
                                    int(count), _ptr(dst_dev), _ptr(bad_dev),
                                    _stream_handle(stream)), "lbm_gather_rows")


def lbm_net_get_buffer(n, which: int, out) -> int:
    """Copy an intermediate buffer of the last forward / backward pass into the numpy array `out`
    (uint16 holding BF16 bits for the BF16 buffers, float32 otherwise)."""
    return _ck(_lib.lbm_net_get_buffer(n, int(which), _ptr(out), out.nbytes), "lbm_net_get_buffer")


def lbm_net_set_grads(n, host) -> int:
    return _ck(_lib.lbm_net_set_grads(n, _ptr(host)), "lbm_net_set_grads")


def lbm_net_forward(n, x_dev, batch, h, w, y_dev) -> int:
    return _ck(_lib.lbm_net_forward(n, _ptr(x_dev), batch, h, w, _ptr(y_dev)), "lbm_net_forward")


def lbm_net_backward(n, x_dev, t_dev, batch, h, w, loss=None) -> int:
    return _ck(_lib.lbm_net_backward(n, _ptr(x_dev), _ptr(t_dev), batch, h, w, loss),
               "lbm_net_backward")


def lbm_net_adam(n, lr, beta1=0.9, beta2=0.999, eps=1e-8) -> int:
    return _ck(_lib.lbm_net_adam(n, lr, beta1, beta2, eps), "lbm_net_adam")


def lbm_net_train_step(n, x_dev, t_dev, batch, h, w, lr, loss=None) -> int:
    return _ck(_lib.lbm_net_train_step(n, _ptr(x_dev), _ptr(t_dev), batch, h, w, float(lr), loss),
               "lbm_net_train_step")


class Net:
    """The sensor predictor of include/lbm.h (lbm_net_*): 3x3 convolutions cin -> hidden -> hidden
    -> 1.  Parameters are numpy float32 vectors in the order W1, b1, W2, b2, W3, b3; inputs and
    outputs are CUDA tensors (float32, [batch, channels, h, w])."""

    def __init__(self, cin=3, hidden=16, stream=None):
        import torch

        self.n = _lib.lbm_net_create(int(cin), int(hidden))
        if not self.n:
            raise LbmError(_lib.lbm_last_error(), "lbm_net_create")
        self.cin, self.hidden = int(cin), int(hidden)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _ck(_lib.lbm_net_set_stream(self.n, self.stream.cuda_stream), "lbm_net_set_stream")
        self.nparam = _ck(_lib.lbm_net_param_count(self.n), "lbm_net_param_count")

    def set_normalisation(self, shift, scale):
        sh = np.ascontiguousarray(shift, dtype=np.float32)
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        _ck(_lib.lbm_net_set_normalisation(self.n, _ptr(sh), _ptr(sc)), "lbm_net_set_normalisation")

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == self.nparam
        _ck(_lib.lbm_net_set_params(self.n, _ptr(th)), "lbm_net_set_params")

    def params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        _ck(_lib.lbm_net_get_params(self.n, _ptr(out)), "lbm_net_get_params")
        return out

    def grads(self):
        out = np.empty(self.nparam, dtype=np.float32)
        _ck(_lib.lbm_net_get_grads(self.n, _ptr(out)), "lbm_net_get_grads")
        return out

    def set_grads(self, g):
        g = np.ascontiguousarray(g, dtype=np.float32)
        _ck(_lib.lbm_net_set_grads(self.n, _ptr(g)), "lbm_net_set_grads")

    def forward(self, x, out=None):
        import torch

        b, c, hh, ww = x.shape
        y = out if out is not None else torch.empty((b, 1, hh, ww), dtype=torch.float32,
                                                    device=x.device)
        _ck(_lib.lbm_net_forward(self.n, _ptr(x), b, hh, ww, _ptr(y)), "lbm_net_forward")
        return y

    def backward(self, x, t, sync=True):
        b, c, hh, ww = x.shape
        loss = ctypes.c_double()
        _ck(_lib.lbm_net_backward(self.n, _ptr(x), _ptr(t), b, hh, ww,
                                  ctypes.byref(loss) if sync else None), "lbm_net_backward")
        return loss.value if sync else None

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _ck(_lib.lbm_net_adam(self.n, lr, beta1, beta2, eps), "lbm_net_adam")

    def buffer(self, which, shape):
        """An intermediate buffer of the last pass (lbm_net_get_buffer): BF16 buffers come back
        as uint16 arrays of their bits, FP32 ones as float32 arrays of the given shape."""
        bf16 = which in (LBM_NET_BUF_PARAMS_BF16, LBM_NET_BUF_X0, LBM_NET_BUF_A1,
                         LBM_NET_BUF_A2)
        out = np.empty(shape, dtype=np.uint16 if bf16 else np.float32)
        lbm_net_get_buffer(self.n, which, out)
        return out

    def train_step(self, x, t, lr, sync=True):
        b, c, hh, ww = x.shape
        loss = ctypes.c_double()
        _ck(_lib.lbm_net_train_step(self.n, _ptr(x), _ptr(t), b, hh, ww, float(lr),
                                    ctypes.byref(loss) if sync else None), "lbm_net_train_step")
        return loss.value if sync else None

    def close(self):
        if self.n:
            _lib.lbm_net_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            if self.n and _lib is not None:
                self.close()
        except Exception:
            pass


class BlockMesh:
    """Multi-level block mesh on a handle: leaf[nbz, nby, nbx] leaf levels, block edge `edge`."""

    def __init__(self, leaf, edge, lmax, tau_fine, lid=(0.0, 0.0), periodic=0, graphs=True,
                 fusion=None, step_form=None, schedule=None):
        import torch  # noqa: F401  (the caller's CUDA context)

        self.leaf = np.ascontiguousarray(leaf, dtype=np.int8)
        nbz, nby, nbx = self.leaf.shape
        self.nb = (nbx, nby, nbz)
        self.edge, self.lmax = int(edge), int(lmax)
        self.h = lbm_create(LBM_D3Q19, nbx * edge, nby * edge, nbz * edge, float(tau_fine))
        lbm_set_lid(self.h, float(lid[0]), float(lid[1]))
        lbm_set_periodic(self.h, int(periodic))
        lbm_set_graphs(self.h, 1 if graphs else 0)
        if fusion is not None:
            lbm_blocks_set_fusion(self.h, int(fusion))
        if step_form is not None:
            lbm_blocks_set_step_form(self.h, int(step_form))
        if schedule is not None:
            lbm_blocks_set_schedule(self.h, int(schedule))
        self.step(0)

    def cycle_form(self):
        """LBM_SCHEDULE_GRAPH or LBM_SCHEDULE_PERSISTENT: how this mesh runs a cycle."""
        return lbm_blocks_cycle_form(self.h)

    def schedule(self, level):
        return lbm_blocks_schedule(self.h, level)

    def _batch(self, cycles, out):
        return LevelBatch(self.nb[0], self.nb[1], self.nb[2], self.edge, self.lmax,
                          self.leaf.ctypes.data, int(cycles),
                          out.ctypes.data if out is not None else None)

    def step(self, cycles, block_max=False):
        out = np.empty(self.leaf.size) if block_max else None
        lbm_blocks_step(self.h, self._batch(cycles, out))
        return out

    def info(self, level):
        return lbm_blocks_info(self.h, level)

    def block_index(self, bx, by, bz):
        return (bz * self.nb[1] + by) * self.nb[0] + bx

    def get_block(self, level, b):
        n = self.info(level)[0]
        out = np.empty((19, n, n, n))
        lbm_blocks_get(self.h, level, int(b), out)
        return out

    def set_block(self, level, b, f):
        lbm_blocks_set(self.h, level, int(b), np.ascontiguousarray(f, dtype=np.float64))

    def leaf_field(self, level):
        n = self.info(level)[0]
        nbx, nby, nbz = self.nb
        out = np.full((19, nbz * n, nby * n, nbx * n), np.nan)
        for bz in range(nbz):
            for by in range(nby):
                for bx in range(nbx):
                    if self.leaf[bz, by, bx] >= level:
                        out[:, bz * n:(bz + 1) * n, by * n:(by + 1) * n, bx * n:(bx + 1) * n] = \
                            self.get_block(level, self.block_index(bx, by, bz))
        return out

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            if self.h and _lib is not None:
                self.close()
        except Exception:
            pass


def lbm_step_noalloc(lattice, dtype, nx, ny, nz, tau, lid_x, lid_z, periodic, f_in_dev, f_out_dev,
                     block, block_max_dev, stream=None) -> int:
    """One fused step + block sensor maxima that allocates nothing (for callers that may not call
    cudaMalloc); see include/lbm.h."""
    s = stream if stream is None or isinstance(stream, int) else stream.cuda_stream
    return _ck(_lib.lbm_step_noalloc(lattice, dtype, nx, ny, nz, tau, lid_x, lid_z, periodic,
                                     _ptr(f_in_dev), _ptr(f_out_dev), block, _ptr(block_max_dev),
                                     s), "lbm_step_noalloc")


def exported_symbols():
    """Names of the functions declared in include/lbm.h."""
    with open(HEADER) as fh:
        src = fh.read()
    return sorted(set(re.findall(r"LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", src)))


# ----------------------------------------------------------------------------- convenience object
_DTYPE_BYTES = {0: 8, 1: 4, 2: 2, 3: 2}


class Lattice:
    """A lattice handle whose population buffers are PyTorch CUDA tensors (``lbm_attach``).

    ``Lattice(LBM_D3Q19, 256, 256, 256, tau, dtype=LBM_F32)`` -> ``step(n)``, ``sensor(block)``,
    ``flag(T)``, ``flag_top(frac)``, ``populations()``...  Numpy arrays in and out, layout
    (q, nz, ny, nx).
    """

    def __init__(self, lattice, nx, ny, nz, tau, dtype=None, lid=(0.1, 0.0), periodic=0,
                 stream=None, torch_buffers=True, device=None):
        import torch

        self.q = int(lattice)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        if device is not None:
            torch.cuda.set_device(device)
        self.h = lbm_create(self.q, self.nx, self.ny, self.nz, float(tau))
        self.dtype = LBM_F32 if dtype is None else int(dtype)
        lbm_set_dtype(self.h, self.dtype)
        lbm_set_lid(self.h, float(lid[0]), float(lid[1]))
        lbm_set_periodic(self.h, int(periodic))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        lbm_set_stream(self.h, self.stream.cuda_stream)
        self._bufs = None
        if torch_buffers:
            nbytes = lbm_population_bytes(self.h)
            a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            self._bufs = (a, b)
            lbm_attach(self.h, a, b, nbytes)
        lbm_reset(self.h)

    @property
    def shape(self):
        return (self.q, self.nz, self.ny, self.nx)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None
            self._bufs = None

    def __del__(self):
        # at interpreter shutdown the module globals may already be gone; the process exit then
        # releases the device memory anyway
        try:
            if self.h and _lib is not None:
                self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n=1):
        lbm_step(self.h, int(n))

    def sensor(self, block):
        out = np.empty(lbm_nblocks(self.h, block), dtype=np.float64)
        lbm_sensor(self.h, block, out)
        return out

    def flag(self, threshold, block=None):
        if block is not None:
            self.block = block
        out = np.empty(lbm_nblocks(self.h, self.block), dtype=np.int8)
        lbm_flag(self.h, float(threshold), out)
        return out

    def flag_top(self, frac, block=None):
        if block is not None:
            self.block = block
        out = np.empty(lbm_nblocks(self.h, self.block), dtype=np.int8)
        lbm_flag_top(self.h, float(frac), out)
        return out

    _block = 16

    @property
    def block(self):
        return self._block

    @block.setter
    def block(self, b):
        lbm_set_block(self.h, int(b))
        self._block = int(b)

    def levels(self, block, a, b, lmin, lmax, average=False):
        out = np.empty(lbm_nblocks(self.h, block), dtype=np.int8)
        lbm_levels(self.h, block, float(a), float(b), int(lmin), int(lmax),
                   LBM_SENSOR_AVERAGE if average else LBM_SENSOR_LAST, out)
        return out

    def levels_fit(self, block, lmin, lmax, average=False):
        out = np.empty(lbm_nblocks(self.h, block), dtype=np.int8)
        lbm_levels_fit(self.h, block, int(lmin), int(lmax),
                       LBM_SENSOR_AVERAGE if average else LBM_SENSOR_LAST, out)
        return out

    def sensor_average(self, block):
        out = np.empty(lbm_nblocks(self.h, block), dtype=np.float64)
        n = lbm_sensor_average(self.h, block, out)
        return out, n

    def populations(self):
        out = np.empty(self.shape, dtype=np.float64)
        lbm_get_populations(self.h, out)
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == self.shape
        lbm_set_populations(self.h, f)

    def moments(self):
        rho = np.empty((self.nz, self.ny, self.nx))
        u = np.empty((3, self.nz, self.ny, self.nx))
        lbm_get_moments(self.h, rho, u)
        return rho, u

    def sensor_field(self):
        out = np.empty((self.nz, self.ny, self.nx))
        lbm_get_sensor_field(self.h, out)
        return out

    def regrid(self, threshold, coarsen=1, buffer=1, efficiency=0.8, min_width=1, allowed=None,
               nest=1, field=None, max_boxes=1 << 16):
        """Boxes [n, 6] (lo x y z, hi x y z, lattice cells) and the tag grid [tz, ty, tx] of one
        regrid of this lattice from its sensor field (``field``: a CUDA tensor of nz*ny*nx doubles
        to use instead)."""
        r = int(coarsen)
        rs = max(r, 1)  # the shape of the output; the call itself refuses r < 1
        tz = -(-self.nz // rs) if self.nz > 1 else 1
        tshape = (tz, -(-self.ny // rs), -(-self.nx // rs))
        mask = None
        if allowed is not None:
            mask = np.ascontiguousarray(allowed, dtype=np.uint8).reshape(tshape)
        p = RegridParams(r, float(threshold), int(buffer), _ptr(mask), int(nest),
                         float(efficiency), int(min_width))
        tags = np.empty(tshape, dtype=np.uint8)
        boxes = (Box * max(int(max_boxes), 1))()
        n, _ = lbm_regrid(self.h, field, p, boxes, int(max_boxes), tags)
        out = np.array([list(boxes[k].lo) + list(boxes[k].hi) for k in range(n)],
                       dtype=np.int64).reshape(-1, 6)
        return out, tags.astype(bool)

    def conservation(self):
        return lbm_conservation(self.h)

    def raw(self):
        nbytes = lbm_population_bytes(self.h)
        out = np.empty(nbytes, dtype=np.uint8)
        lbm_get_raw(self.h, out, nbytes)
        return out

    def set_raw(self, raw):
        raw = np.ascontiguousarray(raw, dtype=np.uint8)
        lbm_set_raw(self.h, raw, raw.nbytes)

    # slab halos (lbm_set_halo): messages as raw storage bytes
    def set_halo(self, faces):
        lbm_set_halo(self.h, int(faces))

    def halo_export(self, face):
        _, nbytes = lbm_halo_size(self.h)
        out = np.empty(nbytes, dtype=np.uint8)
        lbm_halo_export(self.h, int(face), out)
        return out

    def halo_import(self, face, msg):
        msg = np.ascontiguousarray(msg, dtype=np.uint8)
        _, nbytes = lbm_halo_size(self.h)
        if msg.nbytes != nbytes:
            raise ValueError(f"halo message of {msg.nbytes} bytes, expected {nbytes}")
        lbm_halo_import(self.h, int(face), msg)
