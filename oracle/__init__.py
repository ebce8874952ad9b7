"""Plain FP64 CPU oracle for the fused LBM step and the Knudsen refinement sensor.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The product library (``paper_1507_06767_gb300``)
never imports it, and the two share no code.

The heavy loops live in ``lbm_oracle.c`` (plain C, double precision, one cell at a time); this
module is argument marshalling for it plus the per-block flag rules, which are a handful of
comparisons.  Paper references (arXiv 1507.06767, "Local mesh refinement sensor for the lattice
Boltzmann method"):

* Sec. 2.2, Eqs. (bgklb), (feq_i), (rho), (u): BGK lattice equation, equilibrium, moments;
  collide-and-stream split.
* Eq. (nu_omega): nu = c_s^2 (tau - 1/2), used by ``tau_from_re``.
* Sec. 3.2, Eq. (sensor) / Eq. (kkn): K = (1/q) sum_i |f_i^neq / f_i^eq|.
* Sec. 3.4: the sensor drives refinement; the per-block max and refine/coarsen flags below follow
  the threshold reading (refine if max > T, coarsen if max < T/2, the factor 2 being the growth of
  f^neq under 2x coarsening at fixed Re, Appendix A, Eq. knratio).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SRC_ML = os.path.join(_HERE, "lbm_multilevel.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_EINVAL = -1
ORC_EFEQ = -2

PERIODIC_X, PERIODIC_Y, PERIODIC_Z = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, so IEEE double arithmetic holds)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_ML))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-fopenmp", "-o", tmp, _SRC, _SRC_ML, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("tau", ctypes.c_double), ("lid", ctypes.c_double * 3),
                ("periodic", ctypes.c_int), ("force", ctypes.c_double * 3)]


class _MLDesc(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int * 3), ("edge", ctypes.c_int), ("lmax", ctypes.c_int),
                ("tau_fine", ctypes.c_double), ("lid", ctypes.c_double * 3),
                ("periodic", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(_Params)
            lib.orc_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp,
                                        ctypes.POINTER(ctypes.c_int)]
            lib.orc_step.argtypes = [pp, dp, dp, dp, dp, dp]
            lib.orc_run.argtypes = [pp, dp, dp, ctypes.c_int, dp]
            lib.orc_collide.argtypes = [pp, dp, dp, dp]
            lib.orc_stream_push.argtypes = [pp, dp, dp]
            lib.orc_sensor.argtypes = [pp, dp, dp, dp, dp]
            lib.orc_equilibrium.argtypes = [pp, dp, dp, dp]
            lib.orc_block_max.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, dp]
            lib.orc_conservation.argtypes = [pp, dp, dp, dp]
            lib.orc_step_cells.argtypes = [pp, dp, ctypes.c_longlong,
                                           ctypes.POINTER(ctypes.c_longlong), dp, dp]
            lib.orc_threads.argtypes = []
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.ml_create.argtypes = [ctypes.POINTER(_MLDesc), ctypes.POINTER(ctypes.c_int8),
                                      ctypes.POINTER(ctypes.c_int)]
            lib.ml_create.restype = ctypes.c_void_p
            lib.ml_destroy.argtypes = [ctypes.c_void_p]
            lib.ml_destroy.restype = None
            lib.ml_cycles.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.ml_block_max.argtypes = [ctypes.c_void_p, dp]
            lib.ml_get_block.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp]
            lib.ml_set_block.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp]
            lib.ml_level_info.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), dp]
            lib.ml_set_time_interp.argtypes = [ctypes.c_void_p, ctypes.c_int]
            for name in ("ml_cycles", "ml_block_max", "ml_get_block", "ml_set_block",
                         "ml_level_info", "ml_set_time_interp"):
                getattr(lib, name).restype = ctypes.c_int
            for name in ("orc_threads", "orc_set_threads", "orc_step_cells", "orc_lattice", "orc_step", "orc_run", "orc_collide", "orc_stream_push",
                         "orc_sensor", "orc_equilibrium", "orc_block_max", "orc_conservation"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(status: int, what: str):
    if status == ORC_EFEQ:
        raise FloatingPointError(f"{what}: an equilibrium population is not positive")
    if status != ORC_OK:
        raise ValueError(f"{what}: invalid arguments (status {status})")


def threads() -> int:
    """Threads the oracle's parallel loops use (OpenMP; OMP_NUM_THREADS caps it)."""
    return int(_load().orc_threads())


def set_threads(n: int) -> int:
    """Use n threads in the oracle's parallel loops from now on; returns the previous count."""
    return int(_load().orc_set_threads(int(n)))


def lattice(q: int):
    """Velocity set (c[q,3] int), weights w[q] and opposite index opp[q] of D2Q9 / D3Q19."""
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    opp = np.zeros(q, dtype=np.int32)
    st = _load().orc_lattice(q, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(w),
                             opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    _check(st, "lattice")
    return c, w, opp


def tau_from_re(u_lid: float, L: float, re: float) -> float:
    """tau from Re = u L / nu and nu = c_s^2 (tau - 1/2) (Eq. nu_omega), c_s^2 = 1/3."""
    return 3.0 * u_lid * L / re + 0.5


class Oracle:
    """One lattice configuration.  Fields are numpy float64 arrays of shape (q, nz, ny, nx)."""

    def __init__(self, q, nx, ny, nz=1, tau=0.6, lid=(0.0, 0.0, 0.0), periodic=0,
                 force=(0.0, 0.0, 0.0)):
        self.q, self.nx, self.ny, self.nz = int(q), int(nx), int(ny), int(nz)
        self.tau = float(tau)
        self.lid = tuple(float(v) for v in lid)
        self.periodic = int(periodic)
        self.force = tuple(float(v) for v in force)
        self._p = _Params(self.q, self.nx, self.ny, self.nz, self.tau,
                          (ctypes.c_double * 3)(*self.lid), self.periodic,
                          (ctypes.c_double * 3)(*self.force))
        self.c, self.w, self.opp = lattice(self.q)

    @property
    def shape(self):
        return (self.q, self.nz, self.ny, self.nx)

    @property
    def cell_shape(self):
        return (self.nz, self.ny, self.nx)

    def rest(self) -> np.ndarray:
        """The initial cavity state: every population at its weight (rho = 1, u = 0)."""
        f = np.empty(self.shape, dtype=np.float64)
        f[:] = self.w[:, None, None, None]
        return f

    def _field(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == self.shape, (f.shape, self.shape)
        return f

    def step(self, fs, sensor=False, moments=False):
        """One pull step from the post-collision field fs.  Returns (fs_new, K, rho, u) with K / rho /
        u None unless asked for (they describe the pre-collision state of this step)."""
        fs = self._field(fs)
        out = np.empty_like(fs)
        K = np.empty(self.cell_shape) if sensor else None
        rho = np.empty(self.cell_shape) if moments else None
        u = np.empty((3,) + self.cell_shape) if moments else None
        _check(_load().orc_step(ctypes.byref(self._p), _ptr(fs), _ptr(out), _ptr(K), _ptr(rho),
                                _ptr(u)), "step")
        return out, K, rho, u

    def step_cells(self, fs, cells):
        """One pull step evaluated only at the cells with the given linear indices
        ((z*ny + y)*nx + x).  Returns (f_out[len(cells), q], K[len(cells)])."""
        fs = self._field(fs)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.empty((len(cells), self.q))
        K = np.empty(len(cells))
        _check(_load().orc_step_cells(ctypes.byref(self._p), _ptr(fs), len(cells),
                                      cells.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                      _ptr(out), _ptr(K)), "step_cells")
        return out, K

    def run(self, fs, n, sensor_last=False):
        """n pull steps; returns (fs_n, K of the last step or None)."""
        fs = self._field(fs).copy()
        scratch = np.empty_like(fs)
        K = np.empty(self.cell_shape) if sensor_last else None
        _check(_load().orc_run(ctypes.byref(self._p), _ptr(fs), _ptr(scratch), int(n), _ptr(K)),
               "run")
        return fs, K

    def collide(self, f, sensor=False):
        """Push form: collide a pre-collision field.  Returns (f_out, K or None)."""
        f = self._field(f)
        out = np.empty_like(f)
        K = np.empty(self.cell_shape) if sensor else None
        _check(_load().orc_collide(ctypes.byref(self._p), _ptr(f), _ptr(out), _ptr(K)), "collide")
        return out, K

    def stream_push(self, f_out):
        """Push form: stream a post-collision field, bouncing back at the walls."""
        f_out = self._field(f_out)
        nxt = np.full_like(f_out, np.nan)
        _check(_load().orc_stream_push(ctypes.byref(self._p), _ptr(f_out), _ptr(nxt)), "stream")
        return nxt

    def sensor(self, f):
        """Sensor K, rho and u of a pre-collision field."""
        f = self._field(f)
        K = np.empty(self.cell_shape)
        rho = np.empty(self.cell_shape)
        u = np.empty((3,) + self.cell_shape)
        _check(_load().orc_sensor(ctypes.byref(self._p), _ptr(f), _ptr(K), _ptr(rho), _ptr(u)),
               "sensor")
        return K, rho, u

    def equilibrium(self, rho, u):
        rho = np.ascontiguousarray(np.broadcast_to(rho, self.cell_shape), dtype=np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (3,) + self.cell_shape), dtype=np.float64)
        f = np.empty(self.shape)
        _check(_load().orc_equilibrium(ctypes.byref(self._p), _ptr(rho), _ptr(u), _ptr(f)),
               "equilibrium")
        return f

    def conservation(self, f):
        f = self._field(f)
        m = ctypes.c_double()
        j = np.zeros(3)
        _check(_load().orc_conservation(ctypes.byref(self._p), _ptr(f), ctypes.byref(m), _ptr(j)),
               "conservation")
        return m.value, j


def block_max(K: np.ndarray, b: int) -> np.ndarray:
    """Per-block max of a per-cell field K[nz,ny,nx] over blocks of edge b (partial blocks at the
    high ends).  Returns a flat array, x fastest; NaN propagates."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    if K.ndim == 2:
        K = K[None]
    nz, ny, nx = K.shape
    bz = 1 if nz == 1 else b
    nb = -(-nx // b) * -(-ny // b) * -(-nz // bz)
    out = np.empty(nb)
    if nz == 1:
        st = _load().orc_block_max(_ptr(K), nx, ny, 1, b, _ptr(out))
    else:
        st = _load().orc_block_max(_ptr(K), nx, ny, nz, b, _ptr(out))
    _check(st, "block_max")
    return out


def flags_threshold(maxima, T: float) -> np.ndarray:
    """Refine (+1) if max > T, coarsen (-1) if max < T/2, keep (0) otherwise.  A NaN max counts as
    +inf, so it is refined.  Comparisons are made in double precision."""
    out = np.zeros(len(maxima), dtype=np.int8)
    for k, m in enumerate(maxima):
        m = float(m)
        if math.isnan(m) or m > T:
            out[k] = 1
        elif m < T / 2.0:
            out[k] = -1
    return out


def top_count(frac: float, n: int) -> int:
    """Number of blocks refined by the top-fraction rule: ceil(frac * n), clamped to [0, n]."""
    k = math.ceil(frac * n)
    return max(0, min(n, k))


def flags_top(maxima, frac: float) -> np.ndarray:
    """Refine (+1) the ceil(frac * n) largest blocks, keep (0) the rest.  Order: max descending,
    block index ascending on ties; a NaN max counts as +inf."""
    n = len(maxima)
    k = top_count(frac, n)
    keyed = []
    for idx, m in enumerate(maxima):
        m = float(m)
        keyed.append((math.inf if math.isnan(m) else m, idx))
    order = sorted(keyed, key=lambda t: (-t[0], t[1]))
    out = np.zeros(n, dtype=np.int8)
    for _, idx in order[:k]:
        out[idx] = 1
    return out


def flags_agree(flags, ref_maxima, rule: str, param: float, rel_tol: float):
    """Compare flags computed elsewhere with the oracle's flags on its own maxima, ignoring blocks
    whose oracle maximum lies within rel_tol (relative) of a decision boundary: T and T/2 for the
    threshold rule, the k-th largest value for the top-fraction rule.  Returns (ok, n_compared,
    n_excluded)."""
    ref_maxima = np.asarray(ref_maxima, dtype=np.float64)
    flags = np.asarray(flags)
    if rule == "threshold":
        ref = flags_threshold(ref_maxima, param)
        bounds = [param, param / 2.0]
    else:
        ref = flags_top(ref_maxima, param)
        k = top_count(param, len(ref_maxima))
        vals = np.where(np.isnan(ref_maxima), np.inf, ref_maxima)
        kth = np.sort(vals)[::-1][k - 1] if 0 < k <= len(vals) else None
        bounds = [] if kth is None else [kth]
    near = np.zeros(len(ref), dtype=bool)
    for b in bounds:
        if np.isfinite(b):
            near |= np.abs(ref_maxima - b) <= rel_tol * abs(b)
    keep = ~near
    ok = bool(np.array_equal(flags[keep], ref[keep]))
    return ok, int(keep.sum()), int(near.sum())


def levels_affine(maxima, a: float, b: float, lmin: int, lmax: int) -> np.ndarray:
    """Refinement level per block from its sensor maximum (Sec. 3.4, Eqs. phi and l):
    phi = log2(K), l = clamp(floor(a * phi + b), lmin, lmax).  The paper writes [a phi] for the
    integral part; the reading here is the floor, with an offset b (b = 0 is the paper's form).
    K <= 0 gives lmin, NaN gives lmax (a NaN block is refined, as by the flag rules)."""
    out = np.empty(len(maxima), dtype=np.int8)
    for k, m in enumerate(maxima):
        m = float(m)
        if math.isnan(m):
            out[k] = lmax
        elif m <= 0.0:
            out[k] = lmin
        else:
            v = math.floor(a * math.log2(m) + b)
            out[k] = max(lmin, min(lmax, v))
    return out


def levels_fit_params(maxima, lmin: int, lmax: int):
    """The scale a and offset b that map the encountered range of phi = log2(K) (blocks with a
    finite K > 0) linearly onto [lmin, lmax + 1): the normalised phi of the paper's figures
    (Sec. 4, 'normalized phi'), phi_n = (phi - phi_min) / (phi_max - phi_min), gives
    l = lmin + floor(phi_n (lmax - lmin + 1)), clamped.  Returns (a, b) or None if fewer than two
    distinct values exist (all blocks then get lmin)."""
    phis = [math.log2(float(m)) for m in maxima if float(m) > 0.0 and math.isfinite(float(m))]
    if not phis:
        return None
    lo, hi = min(phis), max(phis)
    if not hi > lo:
        return None
    a = float(lmax - lmin + 1) / (hi - lo)
    b = float(lmin) - a * lo
    return a, b


def levels_fit(maxima, lmin: int, lmax: int) -> np.ndarray:
    ab = levels_fit_params(maxima, lmin, lmax)
    if ab is None:
        out = np.full(len(maxima), lmin, dtype=np.int8)
        out[np.isnan(np.asarray(maxima, dtype=np.float64))] = lmax
        return out
    return levels_affine(maxima, ab[0], ab[1], lmin, lmax)


def levels_agree(levels, maxima, a, b, rel_band: float):
    """Compare levels computed elsewhere with levels_affine, ignoring blocks whose a*log2(K) + b lies
    within rel_band of an integer (log2 implementations may differ in the last bit)."""
    ref = levels_affine(maxima, a, b, -128, 127)
    keep = np.ones(len(ref), dtype=bool)
    for k, m in enumerate(maxima):
        m = float(m)
        if m > 0.0 and math.isfinite(m):
            v = a * math.log2(m) + b
            if abs(v - round(v)) <= rel_band * max(1.0, abs(v)):
                keep[k] = False
    return keep


class MultiLevel:
    """Multi-level block-structured D3Q19 mesh (refinement ratio 2, acoustic scaling, level
    sub-cycling, f^neq rescaling at level interfaces; lbm_multilevel.c states the reading of
    Sec. 2.1 / Sec. 5.2 it implements).  leaf[nbz, nby, nbx] holds the leaf level per physical
    block of edge `edge` finest cells."""

    def __init__(self, leaf, edge, lmax, tau_fine, lid=(0.0, 0.0, 0.0), periodic=0):
        leaf = np.ascontiguousarray(leaf, dtype=np.int8)
        assert leaf.ndim == 3
        self.leaf = leaf
        self.nb = (leaf.shape[2], leaf.shape[1], leaf.shape[0])
        self.edge, self.lmax = int(edge), int(lmax)
        d = _MLDesc((ctypes.c_int * 3)(*self.nb), self.edge, self.lmax, float(tau_fine),
                    (ctypes.c_double * 3)(*[float(v) for v in lid]), int(periodic))
        st = ctypes.c_int()
        self._h = _load().ml_create(ctypes.byref(d), leaf.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int8)), ctypes.byref(st))
        if not self._h:
            raise ValueError(f"multi-level mesh rejected (status {st.value})")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ml_destroy(self._h)
            self._h = None

    def level_info(self, l):
        n = ctypes.c_int()
        tau = ctypes.c_double()
        _check(_load().ml_level_info(self._h, l, ctypes.byref(n), ctypes.byref(tau)), "info")
        return n.value, tau.value

    def set_time_interp(self, mode):
        """Test hook: 0 (default) interpolates a fine level's ghosts linearly in time (theta = 0
        and 1/2 on its two sub-steps); 1 plants the mistake theta = 0 on both (the coarse level
        frozen over its step), for the pin that shows the test can tell them apart."""
        _check(_load().ml_set_time_interp(self._h, int(mode)), "set_time_interp")

    def cycles(self, c):
        _check(_load().ml_cycles(self._h, int(c)), "cycles")

    def block_max(self):
        out = np.empty(self.leaf.size)
        _check(_load().ml_block_max(self._h, _ptr(out)), "block_max")
        return out

    def block_index(self, bx, by, bz):
        return (bz * self.nb[1] + by) * self.nb[0] + bx

    def get_block(self, level, b):
        n, _ = self.level_info(level)
        out = np.empty((19, n, n, n))
        _check(_load().ml_get_block(self._h, level, int(b), _ptr(out)), "get_block")
        return out

    def set_block(self, level, b, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        _check(_load().ml_set_block(self._h, level, int(b), _ptr(f)), "set_block")

    def leaf_field(self, level):
        """Assemble the level's populations over the whole domain (blocks where the level exists;
        NaN elsewhere): shape (19, nz, ny, nx) in level-l cells."""
        n, _ = self.level_info(level)
        nbx, nby, nbz = self.nb
        out = np.full((19, nbz * n, nby * n, nbx * n), np.nan)
        for bz in range(nbz):
            for by in range(nby):
                for bx in range(nbx):
                    if self.leaf[bz, by, bx] >= level:
                        out[:, bz * n:(bz + 1) * n, by * n:(by + 1) * n, bx * n:(bx + 1) * n] = \
                            self.get_block(level, self.block_index(bx, by, bz))
        return out
