"""Regridding of one refinement level from the Knudsen sensor: tagging, buffer cells, proper
nesting and Berger-Rigoutsos clustering.  Plain numpy / Python, integers only after tagging.

TEST INFRASTRUCTURE ONLY: imported by the test suite (and ``bench.py``'s CPU legs) alone; the
product library never imports it and shares no code with it.

Paper: arXiv 1507.06767, Sec. 5.2 (dynamic refinement of the 3-D cavity in AMROC): the sensor is
evaluated and the mesh reorganised at the start of every level-0 step; cells flagged by the
sensor get one layer of buffer cells; refinement boxes must hold at least 80 % flagged cells and
are subdivided otherwise; every refinement lies inside the next coarser level with at least one
row of coarse buffer cells (proper nesting).  The paper does not print the clustering algorithm
(it defers to AMROC); the reading here is the point-clustering method of Berger and Rigoutsos
(1991): signatures, holes, inflection points of the signature's second difference, bisection.

Reading, step by step (all coordinates in tag cells, arrays indexed [z, y, x], box axes 0 = x,
1 = y, 2 = z, boxes half-open):

1. tags: a tag cell is r x r (x r along z when nz > 1) lattice cells, cut at the high ends; it is
   tagged if the sensor exceeds the threshold (K > T) in one of its cells or one of them is NaN.
2. buffer: a tag cell is tagged if a tagged cell lies within Chebyshev distance b (periodic axes
   wrap, the domain edge stops the buffer elsewhere).
3. proper nesting: with a mask A of the tag cells that the coarser level covers, a cell stays
   tagged only if every cell within Chebyshev distance `nest` is in A; positions beyond a
   non-periodic domain edge count as covered (no buffer is needed at a physical boundary).
4. clustering, for each box (starting from the whole tag grid):
   a. signatures: the number of tags in each slab normal to each axis;
   b. shrink the box to the bounding box of its tags (drop empty end slabs); an empty box is dropped;
   c. accept the box if tags / volume >= efficiency;
   d. else split it at a hole (an empty slab), the one nearest its axis's centre (least |2p - L|;
      ties: longer axis, lower axis, lower position), the hole starting the upper piece;
   e. else split at the strongest inflection: a strict sign change between second differences
      D[i] = s[i-1] - 2 s[i] + s[i+1] and D[i+1], split between slabs i and i+1, strength
      |D[i+1] - D[i]| (ties: nearer the centre, longer axis, lower axis, lower position);
   f. else bisect the longest axis (ties: lower axis) at floor(L / 2);
   g. a split is admissible only if both pieces are at least `min_width` slabs long; with none
      admissible the box is accepted as it is.
   The boxes are returned sorted by (lo_z, lo_y, lo_x).
"""
from __future__ import annotations

import itertools

import numpy as np


def _as3(a):
    a = np.asarray(a)
    return a[None] if a.ndim == 2 else a


def tag_cells(K, T: float, r: int = 1) -> np.ndarray:
    """Step 1: boolean tag grid [tz, ty, tx] of the per-cell field K[nz, ny, nx] (or [ny, nx])."""
    K = _as3(np.asarray(K, dtype=np.float64))
    nz, ny, nx = K.shape
    rz = r if nz > 1 else 1
    tz, ty, tx = -(-nz // rz), -(-ny // r), -(-nx // r)
    hit = (K > T) | np.isnan(K)
    pad = np.zeros((tz * rz, ty * r, tx * r), dtype=bool)
    pad[:nz, :ny, :nx] = hit
    return pad.reshape(tz, rz, ty, r, tx, r).any(axis=(1, 3, 5))


def _shifted(a, d, periodic, fill):
    """s[p] = a[p - d] (d = (dz, dy, dx)); out-of-range sources wrap on periodic axes, else
    read `fill`."""
    out = np.full(a.shape, fill, dtype=bool)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    rolled = a
    for ax in range(3):
        n = a.shape[ax]
        k = d[ax]
        per = bool(periodic & (1 << (2 - ax)))  # array axis 0 = z (bit 4), 2 = x (bit 1)
        if per:
            rolled = np.roll(rolled, k, axis=ax)
            continue
        if abs(k) >= n:
            return out
        if k >= 0:
            dst[ax] = slice(k, n)
            src[ax] = slice(0, n - k)
        else:
            dst[ax] = slice(0, n + k)
            src[ax] = slice(-k, n)
    out[tuple(dst)] = rolled[tuple(src)]
    return out


def dilate(tags, b: int, periodic: int = 0) -> np.ndarray:
    """Step 2: every cell within Chebyshev distance b of a tagged cell."""
    tags = _as3(np.asarray(tags, dtype=bool))
    out = tags.copy()
    for d in itertools.product(range(-b, b + 1), repeat=3):
        out |= _shifted(tags, d, periodic, False)
    return out


def erode(allowed, nest: int, periodic: int = 0) -> np.ndarray:
    """Step 3's eroded mask: cells whose whole Chebyshev ball of radius `nest` is allowed, the
    outside of a non-periodic edge counting as allowed."""
    allowed = _as3(np.asarray(allowed, dtype=bool))
    out = allowed.copy()
    for d in itertools.product(range(-nest, nest + 1), repeat=3):
        out &= _shifted(allowed, d, periodic, True)
    return out


def _signatures(tags, lo, hi):
    sub = tags[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].astype(np.int64)
    return [sub.sum(axis=(0, 1)), sub.sum(axis=(0, 2)), sub.sum(axis=(1, 2))]


def _choose_split(sig, lens, w):
    """Steps d-g: (axis, p) of the split, p slabs in the lower piece; None if none admissible."""
    ok = lambda L, p: p >= w and L - p >= w  # noqa: E731
    best = None
    for a in range(3):
        L = lens[a]
        for p in range(L):
            if sig[a][p] == 0 and ok(L, p):
                key = (abs(2 * p - L), -L, a, p)
                if best is None or key < best[0]:
                    best = (key, a, p)
    if best is not None:
        return best[1], best[2]
    for a in range(3):
        L = lens[a]
        s = [int(v) for v in sig[a]]
        D = {i: s[i - 1] - 2 * s[i] + s[i + 1] for i in range(1, L - 1)}
        for i in range(1, L - 2):
            if D[i] * D[i + 1] < 0 and ok(L, i + 1):
                p = i + 1
                key = (-abs(D[i + 1] - D[i]), abs(2 * p - L), -L, a, p)
                if best is None or key < best[0]:
                    best = (key, a, p)
    if best is not None:
        return best[1], best[2]
    for a in range(3):
        L = lens[a]
        if ok(L, L // 2):
            key = (-L, a)
            if best is None or key < best[0]:
                best = (key, a, L // 2)
    if best is not None:
        return best[1], best[2]
    return None


def cluster(tags, efficiency: float, min_width: int = 1):
    """Step 4: list of boxes (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z) in tag cells."""
    tags = _as3(np.asarray(tags, dtype=bool))
    tz, ty, tx = tags.shape
    work = [((0, 0, 0), (tx, ty, tz))]
    boxes = []
    while work:
        lo, hi = work.pop()
        sig = _signatures(tags, lo, hi)
        total = int(sig[0].sum())
        if total == 0:
            continue
        lo, hi = list(lo), list(hi)
        for a in range(3):
            nzr = np.nonzero(sig[a])[0]
            first, last = int(nzr[0]), int(nzr[-1])
            sig[a] = sig[a][first:last + 1]
            hi[a] = lo[a] + last + 1
            lo[a] = lo[a] + first
        lens = [hi[a] - lo[a] for a in range(3)]
        vol = lens[0] * lens[1] * lens[2]
        if total >= efficiency * vol:
            boxes.append(tuple(lo) + tuple(hi))
            continue
        split = _choose_split(sig, lens, min_width)
        if split is None:
            boxes.append(tuple(lo) + tuple(hi))
            continue
        a, p = split
        hi_l = list(hi)
        hi_l[a] = lo[a] + p
        lo_u = list(lo)
        lo_u[a] = lo[a] + p
        work.append((tuple(lo_u), tuple(hi)))
        work.append((tuple(lo), tuple(hi_l)))
    boxes.sort(key=lambda b: (b[2], b[1], b[0]))
    return boxes


def regrid(K, T: float, coarsen: int = 1, buffer: int = 1, efficiency: float = 0.8,
           min_width: int = 1, allowed=None, nest: int = 1, periodic: int = 0):
    """Steps 1-4 on a per-cell sensor field.  Returns (boxes in lattice cells as an int array
    [n, 6] = lo_x, lo_y, lo_z, hi_x, hi_y, hi_z, the final tag grid [tz, ty, tx])."""
    K3 = _as3(np.asarray(K, dtype=np.float64))
    nz, ny, nx = K3.shape
    tags = dilate(tag_cells(K3, T, coarsen), buffer, periodic)
    if allowed is not None:
        allowed = _as3(np.asarray(allowed, dtype=bool))
        assert allowed.shape == tags.shape, (allowed.shape, tags.shape)
        tags &= erode(allowed, nest, periodic)
    rz = coarsen if nz > 1 else 1
    scale = (coarsen, coarsen, rz)
    ext = (nx, ny, nz)
    out = []
    for b in cluster(tags, efficiency, min_width):
        out.append([b[a] * scale[a] for a in range(3)] +
                   [min(b[3 + a] * scale[a], ext[a]) for a in range(3)])
    return np.array(out, dtype=np.int64).reshape(-1, 6), tags
