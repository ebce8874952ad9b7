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
* a standing sound wave through a refined band follows the closed form of the damped linear
  wave, with an error that falls at second order with the linear temporal interpolation of the
  coarse level and only at first order with the planted mistake of a coarse level frozen over its
  step (theta = 0 on both fine sub-steps);
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


def _damped_sound(x, t, k, nu, eps, phase):
    """Standing sound wave of the linearised isothermal lattice fluid from rest: density
    1 + eps sin(k x + phase) at t = 0, u = 0.  With shear viscosity nu = c_s^2 (tau - 1/2)
    (Eq. nu_omega) and the BGK bulk viscosity 2 nu / 3, the longitudinal viscosity is 2 nu and
    the amplitude obeys T'' + 2 nu k^2 T' + c_s^2 k^2 T = 0, T(0) = eps, T'(0) = 0."""
    cs2 = 1.0 / 3.0
    om = math.sqrt(cs2 * k * k - (nu * k * k) ** 2)
    g = nu * k * k
    return 1.0 + eps * np.sin(k * x + phase) * math.exp(-g * t) * (math.cos(om * t)
                                                                     + g / om * math.sin(om * t))


def _sound_wave(edge, cycles, frozen=False, tau_f=0.8, eps=1e-4, nbx=8):
    """A standing sound wave along x through a periodic box whose middle half is refined (two
    interfaces, at velocity antinodes).  Returns the largest density error against the closed
    form on the fine level's cells and on the coarse level's leaf cells, relative to eps."""
    c, w, _ = O.lattice(19)
    leaf = np.zeros((1, 1, nbx), np.int8)
    leaf[0, 0, nbx // 4:3 * nbx // 4] = 1
    m = O.MultiLevel(leaf, edge, 1, tau_f, periodic=7)
    m.set_time_interp(1 if frozen else 0)
    k, phase = 2 * math.pi / (nbx * edge), math.pi / 2
    for level in (0, 1):
        n, _ = m.level_info(level)
        h = 2 ** (1 - level)
        for bx in range(nbx):
            if leaf[0, 0, bx] < level:
                continue
            x = (bx * n + np.arange(n) + 0.5) * h
            rho = np.broadcast_to(1.0 + eps * np.sin(k * x + phase), (n, n, n))
            # equilibrium at rest: w_i rho
            m.set_block(level, m.block_index(bx, 0, 0), w[:, None, None, None] * rho[None])
    m.cycles(cycles)
    nu, t = (tau_f - 0.5) / 3.0, 2 * cycles  # time in finest steps
    errs = []
    for level in (0, 1):
        n, _ = m.level_info(level)
        rho = m.leaf_field(level).sum(0)
        x = (np.arange(rho.shape[2]) + 0.5) * 2 ** (1 - level)
        leaf_cells = leaf[0, 0].repeat(n) == level
        ref = _damped_sound(x[leaf_cells], t, k, nu, eps, phase)
        errs.append(float(np.abs(rho[:, :, leaf_cells] - ref).max() / eps))
    return errs


def test_sound_wave_pins_the_closed_form_on_the_uniform_lattice():
    """The closed form used by the temporal-interpolation pin, checked on the uniform oracle
    lattice (no interface): a quarter period of the 64-cell wave within 1e-4 of its amplitude."""
    c, w, _ = O.lattice(19)
    n, tau, eps = 64, 0.8, 1e-4
    k = 2 * math.pi / n
    u = O.Oracle(19, n, 4, 4, tau, periodic=7)
    x = np.arange(n) + 0.5
    rho = np.broadcast_to(1.0 + eps * np.cos(k * x), (4, 4, n))
    f, _ = u.run(w[:, None, None, None] * rho[None], 28)
    ref = _damped_sound(x, 28, k, (tau - 0.5) / 3.0, eps, math.pi / 2)
    assert np.abs(f.sum(0) - ref[None, None, :]).max() / eps < 1e-4


def test_temporal_interpolation_is_second_order():
    """Linear temporal interpolation of the coarse level (theta = 0 and 1/2 on the fine level's two
    sub-steps, Sec. 5.2) against the planted mistake theta = 0 on both.  In a sound wave the state
    at an interface changes at first order within one coarse step (omega dt_c = c_s k dx_c under
    acoustic scaling), so a coarse level frozen over its step leaves a first-order error while the
    linear reading keeps the coupling second order.  A quarter period of the wave, at 64 and 128
    finest cells per wavelength: the linear reading's error falls by >= 3.5x on both levels and
    stays below 2e-3 of the amplitude; the frozen one falls by < 2.2x and is > 5x larger."""
    lin8, lin16 = _sound_wave(8, 14), _sound_wave(16, 28)
    frz8, frz16 = _sound_wave(8, 14, frozen=True), _sound_wave(16, 28, frozen=True)
    for a, b in zip(lin8, lin16):
        assert a / b > 3.5, (lin8, lin16)
    assert max(lin16) < 2e-3, lin16
    assert frz8[1] / frz16[1] < 2.2, (frz8, frz16)
    assert frz16[1] > 5 * max(lin16), (frz16, lin16)


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
