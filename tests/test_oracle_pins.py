"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage of arXiv 1507.06767 it rests on.  The pins are chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign, a swapped index or axis, a wrong tau)
breaks at least one of them:

* lattice tables: isotropy conditions of the velocity sets (needed for Eq. feq_i to recover
  Eqs. ns1-ns2);
* collision: exact mass and momentum invariance per cell (Eqs. rho, u);
* cavity: exact total mass conservation of bounce-back + moving lid;
* uniform equilibrium: zero sensor (Eq. sensor with f^neq = 0);
* pre/post relation: the post-collision f^neq is (1 - 1/tau) times the pre-collision one;
* Couette: exact linear profile (half-way bounce-back) and sensor = CE closed form (Eq. generalf1);
* Poiseuille: exact parabola at the BGK "magic" tau, with nu from Eq. nu_omega;
* Taylor-Green: viscous decay rate nu = c_s^2 (tau - 1/2) (Eq. nu_omega), 2nd-order convergence,
  and the sensor against the CE closed form;
* brute force: pull form == push form bit for bit (the collide-and-stream split of Sec. 2.2), and a
  hand-worked 1x1 cavity stream;
* block max / flags: brute force and hand-made cases.
"""
import math

import numpy as np
import pytest

import oracle as O
from tests import seeded

EPS = np.finfo(np.float64).eps


def perturbed(o, seed, amp=0.02):
    d = seeded.relative_perturbation(seed, o.shape, amp)
    return o.w[:, None, None, None] * (1.0 + d)


# --------------------------------------------------------------------------- lattice tables
@pytest.mark.parametrize("q,d", [(9, 2), (19, 3)])
def test_lattice_isotropy(q, d):
    """Moments of the weights up to 4th order: sum w = 1, odd moments 0, sum w c_a c_b = cs2 delta,
    sum w c_a c_b c_c c_d = cs2^2 (delta delta + ...) -- the conditions under which the truncated
    Maxwellian of Eq. (feq_i) has the moments of Eqs. (rho), (u) and the NS stress."""
    c, w, opp = O.lattice(q)
    cs2 = 1.0 / 3.0
    c = c[:, :d].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose((w[:, None] * c).sum(0), 0.0, atol=1e-16)
    m2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(m2, cs2 * np.eye(d), atol=1e-15)
    m3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(m3, 0.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    I = np.eye(d)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                      + np.einsum("ad,bc->abcd", I, I))
    assert np.allclose(m4, iso, atol=1e-15)
    # velocities are distinct, opposite is an involution pointing the other way
    assert len({tuple(v) for v in c}) == q
    assert np.all(opp[opp] == np.arange(q))
    assert np.all(c[opp] == -c)


@pytest.mark.parametrize("q,d", [(9, 2), (19, 3)])
def test_equilibrium_moments(q, d):
    """The equilibrium must carry the Euler moments the CE expansion builds on (Eqs. rho, u, ns2,
    rho_p): sum feq = rho, sum c feq = rho u, sum c_a c_b feq = rho cs2 delta_ab + rho u_a u_b.
    A dropped or mis-scaled quadratic term of Eq. (feq_i) fails the last one."""
    g = seeded.rng(7)
    o = O.Oracle(q, 3, 2, 1 if q == 9 else 2, tau=0.9)
    rho = 1.0 + g.uniform(-0.1, 0.1, size=o.cell_shape)
    u = g.uniform(-0.1, 0.1, size=(3,) + o.cell_shape)
    if q == 9:
        u[2] = 0.0
    f = o.equilibrium(rho, u)
    c = o.c.astype(float)
    assert np.allclose(f.sum(0), rho, rtol=0, atol=1e-15)
    for a in range(d):
        assert np.allclose(np.einsum("i,i...->...", c[:, a], f), rho * u[a], rtol=0, atol=1e-15)
        for b in range(d):
            pi = np.einsum("i,i,i...->...", c[:, a], c[:, b], f)
            expect = rho * u[a] * u[b] + (rho / 3.0 if a == b else 0.0)
            assert np.allclose(pi, expect, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------- collision invariants
@pytest.mark.parametrize("q,dims", [(9, (7, 5, 1)), (19, (5, 4, 3))])
def test_collision_conserves_mass_momentum(q, dims):
    """Eqs. (rho), (u): sum f_eq = sum f and sum c f_eq = sum c f, hence BGK conserves both per cell."""
    o = O.Oracle(q, *dims, tau=0.7)
    f = perturbed(o, seed=11, amp=0.05)
    fo, _ = o.collide(f)
    c = o.c.astype(float)
    for a in range(3):
        before = np.einsum("i,ijkl->jkl", c[:, a], f)
        after = np.einsum("i,ijkl->jkl", c[:, a], fo)
        assert np.abs(after - before).max() <= 8 * EPS * f.sum(0).max()
    assert np.abs(fo.sum(0) - f.sum(0)).max() <= 8 * EPS * f.sum(0).max()
    # and the collision really changed the populations (f^neq was not zero)
    assert np.abs(fo - f).max() > 1e-4


@pytest.mark.parametrize("q,dims,lid", [(9, (16, 16, 1), (0.1, 0, 0)),
                                        (19, (8, 7, 6), (0.1, 0, 0.05))])
def test_cavity_total_mass_exact(q, dims, lid):
    """Bounce-back returns every population to its cell; the lid terms cancel pairwise on every
    lid-adjacent node (edge/corner ghosts on the lid plane move with the lid), so the total mass of
    the closed cavity stays constant to round-off (Sec. 4.1 moving bounce-back)."""
    o = O.Oracle(q, *dims, tau=0.6, lid=lid)
    f = o.rest()
    m0, _ = o.conservation(f)
    steps = 2000 if q == 9 else 400
    f, _ = o.run(f, steps)
    m1, j = o.conservation(f)
    assert abs(m1 - m0) / m0 < 1e-12
    # the lid has set the fluid moving along +x
    assert j[0] > 1e-3


# --------------------------------------------------------------------------- sensor pins
@pytest.mark.parametrize("q,dims,u0", [(9, (6, 5, 1), (0.05, -0.03, 0.0)),
                                       (19, (4, 5, 3), (0.04, 0.02, -0.03))])
def test_uniform_equilibrium_zero_sensor(q, dims, u0):
    """Eq. (sensor) with f = f_eq everywhere: f^neq = 0, so K = 0; a uniform periodic flow stays at
    equilibrium under stream + collide."""
    o = O.Oracle(q, *dims, tau=0.8, periodic=7 if q == 19 else 3)
    f = o.equilibrium(1.02, np.array(u0)[:, None, None, None])
    for _ in range(5):
        f, K, rho, u = o.step(f, sensor=True, moments=True)
        assert K.max() <= 1e-14
        assert np.abs(rho - 1.02).max() < 1e-14
        for a in range(3):
            assert np.abs(u[a] - u0[a]).max() < 1e-15


def test_sensor_pre_post_relation():
    """Collision keeps rho, u (Eqs. rho, u), so f*_i - f_eq_i = (1 - 1/tau)(f_i - f_eq_i): the sensor
    of the post-collision state is |1 - 1/tau| times the pre-collision one."""
    for tau in (0.55, 0.8, 1.7):
        o = O.Oracle(19, 5, 4, 3, tau=tau)
        f = perturbed(o, seed=5, amp=0.03)
        fo, Kpre = o.collide(f, sensor=True)
        Kpost, _, _ = o.sensor(fo)
        assert np.allclose(Kpost, abs(1 - 1 / tau) * Kpre, rtol=1e-11, atol=0)


def test_sensor_hand_value_single_cell():
    """A single D2Q9 cell with known populations: rho, u and K evaluated by hand from Eqs. (rho),
    (u), (feq_i), (sensor) for a state with u = 0, where f_eq_i = w_i rho."""
    o = O.Oracle(9, 1, 1, 1, tau=1.0, periodic=3)
    f = np.array([4, 1, 1, 1, 1, 0.25, 0.25, 0.25, 0.25], float) / 9.0  # rho = 1, u = 0 ... K = 0
    f = f.reshape(9, 1, 1, 1)
    K, rho, u = o.sensor(f)
    assert abs(rho[0, 0, 0] - 1.0) < 1e-15 and np.abs(u).max() < 1e-16 and K.max() < 1e-15
    # move mass from the rest population to the axis ones, symmetric: rho = 1, u = 0 still
    g = f.copy()
    g[0] -= 0.04
    g[1:5] += 0.01
    K, rho, u = o.sensor(g)
    # |f^neq_0|/feq_0 = 0.04/(4/9) = 0.09; each axis: 0.01/(1/9) = 0.09; K = (0.09 + 4*0.09)/9
    assert abs(K[0, 0, 0] - 0.05) < 1e-15


@pytest.mark.parametrize("q,dims,periodic,coef", [
    (9, (4, 8, 1), O.PERIODIC_X, 4.0 / 3.0),
    (19, (3, 8, 3), O.PERIODIC_X | O.PERIODIC_Z, 12.0 / 19.0),
])
def test_couette_profile_and_sensor(q, dims, periodic, coef):
    """Plane Couette between a resting wall (y = -1/2) and the lid (y = ny - 1/2) moving with U:
    half-way bounce-back reproduces the linear profile u_x = U (y + 1/2)/ny exactly.  The CE
    solution (Eq. generalf1) gives the pre-collision f^neq_i = -3 tau w_i c_ix c_iy G, G = U/ny, so
    K = (1/q) sum_i 3 tau |c_ix c_iy| G: (4/3) tau G for D2Q9, (12/19) tau G for D3Q19, with a
    relative correction O(U)."""
    ny = dims[1]
    tau = 1.0
    res = []
    for U in (1e-3, 1e-4):
        o = O.Oracle(q, *dims, tau=tau, lid=(U, 0, 0), periodic=periodic)
        f, _ = o.run(o.rest(), 3000)
        _, K, rho, u = o.step(f, sensor=True, moments=True)
        y = np.arange(ny)
        exact = U * (y + 0.5) / ny
        ux = u[0][:, :, :]
        assert np.abs(ux - exact[None, :, None]).max() < 1e-12 * U / 1e-3
        assert np.abs(u[1]).max() < 1e-15 and np.abs(u[2]).max() < 1e-15
        Kce = coef * tau * U / ny
        res.append(np.abs(K - Kce).max() / Kce)
    # relative error O(U): small, and shrinking ~10x with U
    assert res[0] < 5e-3
    assert res[1] < res[0] / 5


def test_couette_lid_along_z_3d():
    """Same Couette pin with the lid moving along z (periodic x, z): catches a swapped lid component."""
    U, ny, tau = 1e-4, 6, 0.9
    o = O.Oracle(19, 3, ny, 3, tau=tau, lid=(0, 0, U), periodic=O.PERIODIC_X | O.PERIODIC_Z)
    f, _ = o.run(o.rest(), 3000)
    _, K, rho, u = o.step(f, sensor=True, moments=True)
    exact = U * (np.arange(ny) + 0.5) / ny
    assert np.abs(u[2] - exact[None, :, None]).max() < 1e-13
    assert np.abs(u[0]).max() < 1e-16
    Kce = 12.0 / 19.0 * tau * U / ny
    assert np.abs(K - Kce).max() / Kce < 1e-3


def test_poiseuille_magic_tau():
    """Force-driven channel flow, walls at y = -1/2 and ny - 1/2: u(y) = F/(2 rho nu) (y + 1/2)
    (ny - 1/2 - y), nu = c_s^2 (tau - 1/2) (Eq. nu_omega).  With BGK and half-way bounce-back the
    parabola is reproduced to round-off at (tau - 1/2)^2 = 3/16; at other tau the wall slip error
    is O((tau - 1/2)^2 / ny^2).  Guo forcing is oracle-only (the cavity has no body force)."""
    ny, F = 10, 1e-6
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    o = O.Oracle(9, 3, ny, 1, tau=tau, periodic=O.PERIODIC_X, force=(F, 0, 0))
    f, _ = o.run(o.rest(), 12000)
    _, _, rho, u = o.step(f, moments=True)
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny) + 0.5
    exact = F / (2 * nu) * y * (ny - y)
    assert np.abs(u[0, 0, :, 0] - exact).max() / exact.max() < 1e-10
    # a different tau: error visible but small and of the predicted size
    tau2 = 1.2
    o2 = O.Oracle(9, 3, ny, 1, tau=tau2, periodic=O.PERIODIC_X, force=(F, 0, 0))
    f2, _ = o2.run(o2.rest(), 12000)
    _, _, _, u2 = o2.step(f2, moments=True)
    nu2 = (tau2 - 0.5) / 3.0
    exact2 = F / (2 * nu2) * y * (ny - y)
    err2 = np.abs(u2[0, 0, :, 0] - exact2).max() / exact2.max()
    assert 1e-4 < err2 < 8 * ((tau2 - 0.5) ** 2) / ny ** 2 * 4


def _taylor_green(N, u0=0.01, tau=0.8):
    o = O.Oracle(9, N, N, 1, tau=tau, periodic=3)
    k = 2 * math.pi / N
    x = np.arange(N)[None, :]
    y = np.arange(N)[:, None]
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    rho = 1 - 0.75 * u0 ** 2 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    u = np.zeros((3, 1, N, N))
    u[0, 0], u[1, 0] = ux, uy
    f = o.equilibrium(rho[None], u)
    nu = (tau - 0.5) / 3.0
    T = int(round(0.5 / (4 * nu * k * k)))
    ts, E = [], []
    kerr = None
    for t in range(T + 1):
        fn, K, r, uu = o.step(f, sensor=True, moments=True)
        if t % max(1, T // 10) == 0 and t > 0:
            ts.append(t)
            E.append(0.5 * (r * (uu[0] ** 2 + uu[1] ** 2)).sum())
        if t == T // 2:
            Sxx = u0 * k * np.sin(k * x) * np.sin(k * y) * math.exp(-2 * nu * k * k * t)
            Kce = 4.0 / 3.0 * tau * np.abs(Sxx)
            kerr = np.abs(K[0] - Kce).max() / Kce.max()
        f = fn
    slope = np.polyfit(np.array(ts), np.log(np.array(E)), 1)[0]
    return -slope / (4 * k * k) / nu - 1.0, kerr


def test_taylor_green_viscosity_and_sensor():
    """Decaying Taylor-Green vortex: kinetic energy ~ exp(-4 nu k^2 t) with nu = c_s^2 (tau - 1/2)
    (Eq. nu_omega); the fitted nu converges at 2nd order in 1/N.  The sensor follows the CE closed
    form K = (4/3) tau |S_xx| (Eq. generalf1; only the axis directions carry f^neq), with a relative
    correction of the order of the lattice Knudsen number k tau, i.e. first order in 1/N."""
    e16, k16 = _taylor_green(16)
    e32, k32 = _taylor_green(32)
    assert abs(e32) < 2e-3
    assert abs(e16) / abs(e32) > 3.0
    assert k32 < 0.06
    assert 1.6 < k16 / k32 < 2.4


# --------------------------------------------------------------------------- brute force
@pytest.mark.parametrize("q,dims,periodic,lid", [
    (9, (3, 3, 1), 0, (0.1, 0, 0)),
    (9, (4, 4, 1), O.PERIODIC_X, (0.07, 0, 0)),
    (9, (5, 3, 1), O.PERIODIC_Y, (0.0, 0, 0)),
    (19, (4, 4, 4), 0, (0.1, 0, 0.03)),
    (19, (3, 4, 5), O.PERIODIC_Z, (0.05, 0, 0)),
    (19, (4, 3, 2), O.PERIODIC_X | O.PERIODIC_Y, (0.0, 0, 0)),
])
def test_pull_equals_push_bitwise(q, dims, periodic, lid):
    """Sec. 2.2 writes a step as collide then stream (push); the oracle's main form pulls, then
    collides.  Starting from the same post-collision field, n pull steps must equal
    stream, (collide, stream) x (n-1), collide -- bit for bit."""
    o = O.Oracle(q, *dims, tau=0.73, lid=lid, periodic=periodic)
    f0 = perturbed(o, seed=q * 100 + dims[0], amp=0.05)
    for n in (1, 2, 7):
        pull, _ = o.run(f0, n)
        g = o.stream_push(f0)
        for _ in range(n - 1):
            g = o.stream_push(o.collide(g)[0])
        push, _ = o.collide(g)
        assert np.array_equal(pull, push), n
    # streaming alone touches every slot exactly once
    assert not np.isnan(o.stream_push(f0)).any()


def test_hand_stream_one_cell_cavity():
    """A 1x1 D2Q9 cavity: every neighbour is a wall ghost, so each population comes back reversed;
    the ghosts above (y = 1 = ny) are the lid.  By hand (w_diag = 1/36, 2 w c.u / cs2 = 6 w c.u):
    f_4 = f*_2, f_7 (c = (-1,-1)) = f*_5 - U/6, f_8 (c = (1,-1)) = f*_6 + U/6, the rest plainly
    reversed."""
    U = 0.1
    o = O.Oracle(9, 1, 1, 1, tau=1.0, lid=(U, 0, 0))
    fs = (np.arange(9, dtype=float) + 1.0).reshape(9, 1, 1, 1) / 50.0
    g = o.stream_push(fs)
    expect = np.array([fs[0], fs[3], fs[4], fs[1], fs[2], fs[7], fs[8], fs[5] - U / 6,
                       fs[6] + U / 6]).reshape(9)
    assert np.allclose(g.reshape(9), expect, rtol=0, atol=1e-16)
    # tau = 1: the step lands on the equilibrium of the streamed state
    out, _, rho, u = o.step(fs, moments=True)
    assert abs(rho[0, 0, 0] - expect.sum()) < 1e-15
    assert np.allclose(out, o.equilibrium(rho, u), rtol=0, atol=1e-16)


# --------------------------------------------------------------------------- block max / flags
@pytest.mark.parametrize("shape,b", [((1, 13, 17), 4), ((7, 9, 10), 4), ((1, 16, 16), 16),
                                     ((5, 5, 5), 8)])
def test_block_max_brute(shape, b):
    g = seeded.rng(3)
    K = g.uniform(0, 1, size=shape)
    out = O.block_max(K, b)
    nz, ny, nx = shape
    bz = b if nz > 1 else 1
    expect = []
    for z0 in range(0, nz, bz):
        for y0 in range(0, ny, b):
            for x0 in range(0, nx, b):
                expect.append(K[z0:z0 + bz, y0:y0 + b, x0:x0 + b].max())
    assert np.array_equal(out, np.array(expect))
    K2 = K.copy()
    K2.flat[5] = np.nan
    out2 = O.block_max(K2, b)
    assert np.isnan(out2).sum() == 1


def test_flags_threshold_cases():
    T = 1e-3
    m = [2e-3, 1e-3, np.nextafter(1e-3, 1), 5e-4, np.nextafter(5e-4, 0), 7e-4, 0.0, np.nan]
    assert list(O.flags_threshold(m, T)) == [1, 0, 1, 0, -1, 0, -1, 1]


def test_flags_top_cases():
    m = np.array([0.5, 0.1, 0.5, np.nan, 0.2, 0.5, 0.0], dtype=np.float32)
    # k = ceil(0.5 * 7) = 4: NaN first, then the three 0.5's
    assert list(O.flags_top(m, 0.5)) == [1, 0, 1, 1, 0, 1, 0]
    # k = ceil(0.3 * 7) = 3: NaN, then the two lowest-index 0.5's
    assert list(O.flags_top(m, 0.3)) == [1, 0, 1, 1, 0, 0, 0]
    assert O.top_count(0.1, 4096) == 410
    assert list(O.flags_top(m, 0.0)) == [0] * 7
    assert list(O.flags_top(m, 1.0)) == [1] * 7


def test_tau_from_re_paper_cases():
    """Eq. (nu_omega) with Re = u L / nu: the paper's 2D cavity (Re = 1000, u = 0.05, N = 120,
    Sec. 4.1) has nu = 0.006, tau = 0.518; the 128^2 Re = 100 cavity with u = 0.1 has tau = 0.884."""
    assert abs(O.tau_from_re(0.05, 120, 1000) - 0.518) < 1e-12
    assert abs(O.tau_from_re(0.1, 128, 100) - 0.884) < 1e-12
    assert abs(O.tau_from_re(0.1, 256, 1000) - 0.5768) < 1e-12


def test_step_cells_matches_full_step():
    """The sampled-cell evaluation is the same step: it must agree bit for bit with the full step on
    every cell, boundary cells included."""
    o = O.Oracle(19, 6, 5, 4, tau=0.66, lid=(0.1, 0, 0.02), periodic=O.PERIODIC_Z)
    f = perturbed(o, seed=21, amp=0.04)
    full, K, _, _ = o.step(f, sensor=True)
    cells = np.arange(6 * 5 * 4)[::-1].copy()
    out, Kc = o.step_cells(f, cells)
    assert np.array_equal(out, full.reshape(19, -1)[:, cells].T)
    assert np.array_equal(Kc, K.reshape(-1)[cells])


def test_level_map_cases():
    """Sec. 3.4, Eqs. phi and l: phi = log2 K, l = clamp([a phi + b], lmin, lmax) with [.] read as
    the floor.  Powers of two give integer phi, so these cases are exact by hand."""
    m = np.array([2.0 ** -10, 2.0 ** -9, 2.0 ** -4, 2.0 ** -20, 0.0, np.nan, 3 * 2.0 ** -11])
    # a = 0.5, b = 7: phi -10 -> 2, -9 -> 2.5 -> 2, -4 -> 5 -> clamp 4, -20 -> -3 -> clamp 0;
    # log2(3 * 2^-11) = -9.415 -> 2.29 -> 2
    assert list(O.levels_affine(m, 0.5, 7.0, 0, 4)) == [2, 2, 4, 0, 0, 4, 2]
    # fitted: phi in [-20, -4] mapped onto [0, 3): a = 3/16, b = 3.75
    a, b = O.levels_fit_params(m, 0, 2)
    assert abs(a - 3.0 / 16.0) < 1e-15 and abs(b - 3.75) < 1e-15
    # -10 -> 1.875 -> 1; -9 -> 2.0625 -> 2; -4 -> 3 -> clamp 2; -20 -> 0; 0 -> lmin; NaN -> lmax;
    # -9.415 -> 1.985 -> 1
    assert list(O.levels_fit(m, 0, 2)) == [1, 2, 2, 0, 0, 2, 1]
    # one distinct value: nothing to scale, all lmin (NaN still refines)
    assert list(O.levels_fit(np.array([0.25, 0.25, np.nan]), 1, 3)) == [1, 1, 3]
