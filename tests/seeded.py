"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module only draws random numbers (and encodes draws in the 16-bit storage formats); it holds
none of the lattice Boltzmann arithmetic.  Callers turn the draws into populations themselves
(f_i = w_i (1 + a * delta_i) with the oracle's weights).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def relative_perturbation(seed: int, shape, amplitude: float) -> np.ndarray:
    """Uniform draws in [-amplitude, amplitude] of the given shape (float64)."""
    return rng(seed).uniform(-amplitude, amplitude, size=shape)


def smooth_perturbation(seed: int, shape, amplitude: float, modes: int = 3) -> np.ndarray:
    """A sum of a few random low Fourier modes along each lattice axis, per leading index, scaled to
    peak |value| <= amplitude.  shape = (q, nz, ny, nx)."""
    g = rng(seed)
    q, nz, ny, nx = shape
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    out = np.zeros(shape)
    for i in range(q):
        acc = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kx, ky, kz = g.integers(0, 3, size=3)
            ph = g.uniform(0, 2 * np.pi, size=3)
            acc += (np.cos(2 * np.pi * kx * x / nx + ph[0]) * np.cos(2 * np.pi * ky * y / ny + ph[1])
                    * np.cos(2 * np.pi * kz * z / max(nz, 1) + ph[2]))
        peak = np.abs(acc).max()
        out[i] = acc * (amplitude / peak if peak > 0 else 0.0)
    return out


def block_maxima(seed: int, n: int, ties: int = 0, nans: int = 0, near=None) -> np.ndarray:
    """float32 per-block maxima drawn log-uniformly in [1e-5, 1e-1], with `ties` entries repeated,
    `nans` NaN entries and, if `near` = (T, count), `count` entries within 1 ulp-ish of T and T/2."""
    g = rng(seed)
    v = np.exp(g.uniform(np.log(1e-5), np.log(1e-1), size=n)).astype(np.float32)
    if ties and n > 1:
        src = g.integers(0, n, size=ties)
        dst = g.integers(0, n, size=ties)
        v[dst] = v[src]
    if nans:
        v[g.choice(n, size=min(nans, n), replace=False)] = np.nan
    if near is not None:
        T, count = near
        idx = g.choice(n, size=min(count, n), replace=False)
        for j, k in enumerate(idx):
            base = np.float32(T if j % 2 == 0 else T / 2)
            v[k] = np.nextafter(base, np.float32(np.inf if j % 4 < 2 else 0), dtype=np.float32)
            if j % 3 == 0:
                v[k] = base
    return v


def rng_for(*key) -> np.random.Generator:
    """Generator seeded by a tuple of names and integers (stable across runs and machines)."""
    import zlib

    return rng(zlib.crc32(repr(key).encode()))


def blob_field(seed: int, shape, blobs: int = 6, background=(1e-5, 1e-3), peak=(1e-2, 1e-1)):
    """A positive per-cell field [nz, ny, nx] shaped like a refinement sensor: log-uniform
    background noise plus a few Gaussian bumps of log-uniform height and radius 1..shape/6."""
    g = rng(seed)
    nz, ny, nx = shape
    f = np.exp(g.uniform(np.log(background[0]), np.log(background[1]), size=shape))
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(blobs):
        c = [g.uniform(0, n) for n in shape]
        r = g.uniform(1.0, max(1.5, max(shape) / 6.0))
        h = np.exp(g.uniform(np.log(peak[0]), np.log(peak[1])))
        d2 = (zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2
        f += h * np.exp(-d2 / (2.0 * r * r))
    return f


def uniform_arrays(seed: int, shapes, limits):
    """One uniform draw in [-lim, lim] per (shape, lim) pair, in order (e.g. network weights)."""
    g = rng(seed)
    return [g.uniform(-lim, lim, size=shp) for shp, lim in zip(shapes, limits)]


def stored_deviations16(seed: int, w, n: int, amplitude: float, dtype_name: str,
                        pool: int = 1 << 22) -> np.ndarray:
    """Stored 16-bit populations of a perturbed state in the shifted form f_i - w_i, one row of n
    values per direction: deviations w_i * U(-amplitude, amplitude) rounded to FP16 ("F16S") or
    BF16 ("BF16S", round to nearest even on the upper 16 bits).  Each row repeats a pool of `pool`
    seeded draws (cheap at 10^8 cells and above), started at a seeded offset."""
    g = rng(seed)
    out = np.empty((len(w), n), dtype=np.uint16)
    for i, wi in enumerate(w):
        d = (wi * g.uniform(-amplitude, amplitude, size=pool)).astype(np.float32)
        if dtype_name == "F16S":
            p16 = d.astype(np.float16).view(np.uint16)
        else:
            b = d.view(np.uint32)
            p16 = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)
        p16 = np.roll(p16, int(g.integers(0, pool)))
        out[i] = np.resize(p16, n)
    return out
