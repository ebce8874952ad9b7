"""Pins of the multi-level block-structured oracle (oracle/lbm_multilevel.c), no GPU.

The paper runs its refined meshes with ratio-2 levels under acoustic scaling, sub-cycled and
coupled by interpolation with f^neq rescaling (Sec. 2.1, Sec. 5.2); the oracle file states the
reading.  These pins fix it against what the mathematics fixes:

* one level only: the block mesh with ghost copies is exactly the uniform lattice (bit for bit);
* every block refined: the finest level alone is exactly the uniform fine lattice (bit for bit);
* plane Couette flow across a refinement interface: the steady profile is linear in physical
  coordinates on both levels to round-off -- this needs the Chapman-Enskog rescaling of f^neq
  (Eq. generalf1: f^neq ~ tau dt), the trilinear interpolation and the restriction to be right
  (without the rescaling the error is 15 %);
* a shear wave decaying across an interface follows exp(-nu k^2 t), nu = c_s^2 (tau - 1/2)
  (Eq. nu_omega), with an error that falls at about second order under refinement;
* the fluid at rest stays at rest; unbalanced meshes and tau = 1 are refused.
"""
import math

import numpy as np
import pytest

import oracle as O


def ux_profile(m, level, D):
    n, _ = m.level_info(level)
    h = 2 ** (m.lmax - level)
    f = m.leaf_field(level)
    with np.errstate(invalid="ignore"):
        ux = (f[[1, 7, 9, 11, 13]].sum(0) - f[[2, 8, 10, 12, 14]].sum(0)) / f.sum(0)
    prof = np.array([np.nan if np.isnan(ux[:, j, :]).all() else np.nanmean(ux[:, j, :])
                     for j in range(ux.shape[1])])
    y = (np.arange(len(prof)) + 0.5) * h
    return y, prof


def test_single_level_is_the_uniform_lattice():
    leaf = np.zeros((2, 2, 3), np.int8)
    m = O.MultiLevel(leaf, 4, 0, 0.7, lid=(0.1, 0, 0.02))
    m.cycles(6)
    u = O.Oracle(19, 12, 8, 8, 0.7, lid=(0.1, 0, 0.02))
    fu, _ = u.run(u.rest(), 6)
    assert np.array_equal(m.leaf_field(0), fu)


def test_fully_refined_mesh_is_the_uniform_fine_lattice():
    leaf = np.ones((2, 2, 2), np.int8)
    m = O.MultiLevel(leaf, 4, 1, 0.7, lid=(0.1, 0, 0))
    assert m.level_info(0) == (2, pytest.approx(0.6)) and m.level_info(1) == (4, 0.7)
    m.cycles(3)
    u = O.Oracle(19, 8, 8, 8, 0.7, lid=(0.1, 0, 0))
    fu, _ = u.run(u.rest(), 6)
    assert np.array_equal(m.leaf_field(1), fu)


def test_couette_across_a_refinement_interface():
    U, D = 1e-4, 16.0
    leaf = np.zeros((1, 4, 1), np.int8)
    leaf[:, 2:, :] = 1
    m = O.MultiLevel(leaf, 4, 1, 0.8, lid=(U, 0, 0), periodic=O.PERIODIC_X | O.PERIODIC_Z)
    m.cycles(6000)
    for level, lo, hi in ((0, 0.0, 8.0), (1, 8.0, 16.0)):
        y, prof = ux_profile(m, level, D)
        sel = (y > lo) & (y < hi)
        assert sel.sum() == (4 if level == 0 else 8)
        assert np.abs(prof[sel] - U * y[sel] / D).max() < 1e-9 * U


def _shear_wave(edge):
    tau_f, u0, nby = 0.8, 1e-3, 4
    leaf = np.zeros((1, nby, 1), np.int8)
    leaf[:, nby // 2:, :] = 1
    m = O.MultiLevel(leaf, edge, 1, tau_f, periodic=7)
    D = nby * edge
    for level in (0, 1):
        n, tau = m.level_info(level)
        h = 2 ** (1 - level)
        o = O.Oracle(19, n, n, n, tau)
        for by in range(nby):
            if leaf[0, by, 0] < level:
                continue
            y = (by * n + np.arange(n) + 0.5) * h
            u = np.zeros((3, n, n, n))
            u[0] = (u0 * np.sin(2 * math.pi * y / D))[None, :, None]
            m.set_block(level, m.block_index(0, by, 0), o.equilibrium(1.0, u))
    nu, k = (tau_f - 0.5) / 3.0, 2 * math.pi / D
    cycles = int(round(1.0 / (nu * k * k) / 2))
    m.cycles(cycles)
    exact = math.exp(-nu * k * k * 2 * cycles)
    errs = []
    for level, below in ((0, True), (1, False)):
        y, prof = ux_profile(m, level, D)
        sel = ~np.isnan(prof) & ((y < D / 2) if below else (y >= D / 2))
        amp = (prof[sel] / np.sin(2 * math.pi * y[sel] / D)).mean() / u0
        errs.append(abs(amp / exact - 1))
    return errs


def test_shear_wave_decay_across_an_interface_converges():
    e32 = _shear_wave(8)
    e64 = _shear_wave(16)
    assert max(e64) < 0.025
    assert min(a / b for a, b in zip(e32, e64)) > 2.5


def test_rest_stays_at_rest_on_a_mixed_mesh():
    leaf = np.ones((4, 3, 3), np.int8)
    leaf[0, :, :] = 0
    leaf[2, 1, 1] = 2
    m = O.MultiLevel(leaf, 8, 2, 0.7)
    m.cycles(3)
    for level in (0, 1, 2):
        f = m.leaf_field(level)
        w = O.lattice(19)[1][:, None, None, None]
        assert np.nanmax(np.abs(f - w)) < 1e-15
    assert np.nanmax(m.block_max()) < 1e-14


def test_invalid_meshes_are_refused():
    leaf = np.zeros((1, 1, 3), np.int8)
    leaf[0, 0, 0] = 2  # touches a level-0 block
    with pytest.raises(ValueError):
        O.MultiLevel(leaf, 4, 2, 0.7)
    with pytest.raises(ValueError):  # level-0 tau = 1 (the rescaling divides by tau - 1)
        O.MultiLevel(np.ones((1, 1, 2), np.int8), 4, 1, 1.5)
    with pytest.raises(ValueError):  # edge not divisible into 2 coarse cells
        O.MultiLevel(np.zeros((1, 1, 1), np.int8), 2, 1, 0.7)
