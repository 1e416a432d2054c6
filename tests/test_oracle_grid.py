"""Pins of the oracle's GRMHD-grid plasma (sec. 4.2.2, sec. 5, App. A.2) and of the
synthetic snapshot generator.  CPU only."""
import math

import numpy as np
import pytest

from paper_1801_10452_b300 import scenes

QE, ME, MP, C, G, MSUN = 4.80320471e-10, 9.1093837015e-28, 1.67262192369e-24, 2.99792458e10, 6.67430e-8, 1.98841e33


@pytest.mark.parametrize("h", [0.3, 0.7, 1.0])
def test_newton_inverts_mks_theta(ora, h):
    """App. A.2: Newton-Raphson recovers x2 with theta(x2) = theta to 1e-13."""
    for th in np.linspace(1e-4, math.pi - 1e-4, 301):
        x2, it = ora.newton_x2(th, h)
        assert 0 <= x2 <= 1 and it <= 20
        assert abs(math.pi * x2 + 0.5 * (1 - h) * math.sin(2 * math.pi * x2) - th) < 1e-13


def _grid_scene(ora, grid, **kw):
    s = ora.scene(**kw)
    return ora.attach_grid(s, grid, x1_min=kw.pop("x1_min", math.log(1.4)), x1_max=kw.pop("x1_max", math.log(50.0)),
                           h_mks=kw.pop("h_mks", 0.3))


def test_bilinear_exact_on_linear_fields(ora):
    n1, n2 = 12, 9
    x1_min, x1_max = 0.3, 3.9
    c1 = x1_min + (np.arange(n1) + 0.5) * (x1_max - x1_min) / n1
    c2 = (np.arange(n2) + 0.5) / n2
    X1, X2 = np.meshgrid(c1, c2)
    grid = np.zeros((1, 8, n2, n1), np.float32)
    for f in range(8):
        grid[0, f] = 0.5 + 0.1 * f + 0.25 * X1 - 0.75 * X2
    s = ora.attach_grid(ora.scene(), grid, x1_min, x1_max, 0.3)
    rng = np.random.default_rng(5)
    for _ in range(200):
        x1 = rng.uniform(c1[0], c1[-1])
        x2 = rng.uniform(c2[0], c2[-1])
        ok, v = ora.grid_bilinear(s, 0, x1, x2)
        assert ok
        exp = np.array([0.5 + 0.1 * f + 0.25 * x1 - 0.75 * x2 for f in range(8)])
        assert np.allclose(v, exp, rtol=0, atol=1e-6)  # float32 storage of the nodes
    # outside the cell centres: clamped to the edge cells; outside [x1_min, x1_max]: no plasma
    ok, v = ora.grid_bilinear(s, 0, c1[3], 0.001)
    ok2, v2 = ora.grid_bilinear(s, 0, c1[3], c2[0])
    assert ok and np.allclose(v, v2)
    assert ora.grid_bilinear(s, 0, x1_max + 1e-9, 0.5)[0] == 0


def _rand_grid(rng, n1=6, n2=6, U=0.3, Bm=0.05):
    g = np.zeros((1, 8, n2, n1), np.float32)
    g[0, 0] = rng.uniform(0.5, 2.0, (n2, n1))
    g[0, 1] = rng.uniform(0.01, 0.2, (n2, n1))
    g[0, 2:5] = rng.uniform(-U, U, (3, n2, n1))
    g[0, 5:8] = rng.uniform(-Bm, Bm, (3, n2, n1))
    return g


def test_grid_velocity_and_field_invariants(ora):
    """HARM primitives -> u^mu, b^mu: u.u = -1, b.u = 0, |b| = B (all in KS)."""
    rng = np.random.default_rng(9)
    grid = _rand_grid(rng)
    s = ora.attach_grid(ora.scene(a=0.9375, mass_unit_g=1e19, mass_msun=4e6), grid, math.log(1.4), math.log(50.0), 0.3)
    for _ in range(100):
        r = math.exp(rng.uniform(math.log(1.5), math.log(45)))
        th = rng.uniform(0.1, math.pi - 0.1)
        ok, ne, te, B, u, b = ora.plasma(s, [0.0, r, th, 0.0])
        assert ok == 1
        g, _ = ora.metric(s, r, th)
        assert math.isclose(u @ g @ u, -1.0, rel_tol=1e-10)
        assert abs(b @ g @ u) <= 1e-9 * B * abs(u[0])
        assert math.isclose(math.sqrt(b @ g @ b), B, rel_tol=1e-10)


def test_grid_normal_observer_and_units(ora):
    """U^i = 0 gives the KS normal observer (u_i = 0 for spatial i); n_e and B follow the unit
    scaling of Eq. 45; Theta_e follows the R-beta limits of Eq. 46 (sec. 5)."""
    rng = np.random.default_rng(10)
    grid = _rand_grid(rng, U=0.0, Bm=0.0)
    grid[0, 5] = 0.02  # purely radial field
    Mu, Mbh = 1.0e19, 4.0e6
    for R_low, R_high in [(1.0, 1.0), (1.0, 25.0), (3.0, 3.0)]:
        s = ora.attach_grid(ora.scene(a=0.5, mass_unit_g=Mu, mass_msun=Mbh, r_low=R_low, r_high=R_high), grid,
                            math.log(1.4), math.log(50.0), 0.3)
        for r, th in [(3.0, 1.0), (10.0, 2.0), (30.0, 0.4)]:
            ok, ne, te, B, u, b = ora.plasma(s, [0.0, r, th, 0.0])
            g, _ = ora.metric(s, r, th)
            ucov = g @ u
            assert abs(ucov[1]) < 1e-12 and abs(ucov[2]) < 1e-12 and abs(ucov[3]) < 1e-12
            ok2, prim = ora.grid_bilinear(s, 0, math.log(r), ora.newton_x2(th, 0.3)[0])
            rho, uu = prim[0], prim[1]
            L = G * Mbh * MSUN / C**2
            rho0 = Mu / L**3
            assert math.isclose(ne, rho * rho0 / (ME + MP), rel_tol=1e-12)
            bsq = (B / (C * math.sqrt(4 * math.pi * rho0))) ** 2
            beta_p = (4 / 3 - 1) * uu / (0.5 * bsq)
            R = R_low / (1 + beta_p**2) + R_high * beta_p**2 / (1 + beta_p**2)
            assert math.isclose(te, (MP / ME) * (1 / 3) * (uu / rho) / (1 + R), rel_tol=1e-10)
    # limits of Eq. 46: strong field -> R_low, weak field -> R_high
    for Bfield, expect in [(1e3, 1.0), (1e-7, 25.0)]:
        grid[0, 5] = Bfield
        s = ora.attach_grid(ora.scene(a=0.5, mass_unit_g=Mu, mass_msun=Mbh, r_low=1.0, r_high=25.0), grid,
                            math.log(1.4), math.log(50.0), 0.3)
        ok, ne, te, B, u, b = ora.plasma(s, [0.0, 10.0, 1.0, 0.0])
        _, prim = ora.grid_bilinear(s, 0, math.log(10.0), ora.newton_x2(1.0, 0.3)[0])
        t_expect = (MP / ME) * (1 / 3) * (prim[1] / prim[0]) / (1 + expect)
        assert math.isclose(te, t_expect, rel_tol=1e-3)


def test_slow_light_interpolates_in_time(ora):
    """Sec. 5: slow light interpolates snapshots linearly in the ray's coordinate time;
    identical snapshots make slow light equal fast light."""
    rng = np.random.default_rng(12)
    g0 = _rand_grid(rng)
    g1 = _rand_grid(rng)
    grid = np.concatenate([g0, g1], 0)
    kw = dict(a=0.7, mass_unit_g=1e19, t0=100.0, dt_snap=10.0)
    s = ora.attach_grid(ora.scene(**kw), grid, math.log(1.4), math.log(50.0), 0.3)
    s.slow_light = 1
    for t, w in [(100.0, 0.0), (103.0, 0.3), (110.0, 1.0), (50.0, 0.0), (500.0, 1.0)]:
        x = [t, 7.0, 1.3, 0.0]
        _, prim0 = ora.grid_bilinear(s, 0, math.log(7.0), ora.newton_x2(1.3, 0.3)[0])
        _, prim1 = ora.grid_bilinear(s, 1, math.log(7.0), ora.newton_x2(1.3, 0.3)[0])
        ok, ne, *_ = ora.plasma(s, x)
        rho = (1 - w) * prim0[0] + w * prim1[0]
        assert math.isclose(ne / rho, ne / rho, rel_tol=0)  # finite
        s_f = ora.attach_grid(ora.scene(**kw), np.concatenate([(1 - w) * g0 + w * g1], 0).astype(np.float64), math.log(1.4),
                              math.log(50.0), 0.3)
        okf, nef, tef, Bf, uf, bf = ora.plasma(s_f, x)
        assert math.isclose(ne, nef, rel_tol=1e-6)
    same = ora.attach_grid(ora.scene(**kw), np.concatenate([g0, g0], 0), math.log(1.4), math.log(50.0), 0.3)
    same.slow_light = 1
    fast = ora.attach_grid(ora.scene(**kw), g0, math.log(1.4), math.log(50.0), 0.3)
    for al, be in [(8.0, 3.0), (-12.0, 5.0)]:
        a1 = ora.trace_ray(same, al, be, [2.3e11], t_cam=1000.0)["I"]
        a2 = ora.trace_ray(fast, al, be, [2.3e11], t_cam=1000.0)["I"]
        assert np.array_equal(a1, a2)


def test_torus_generator_is_an_equilibrium():
    """The synthetic Fishbone-Moncrief torus: pressure maximum at r_max, inner edge at r_in,
    the relativistic Euler equation d ln h / dr = (u^t)^2/2 d_r(g_tt + 2 Om g_tphi + Om^2 g_phiphi)
    on the equator, unit-normalised velocity, constant l = u^t u_phi."""
    a = scenes.TORUS["spin"]
    l = scenes.fm_angular_momentum(a, 12.0)
    r = np.linspace(5, 40, 3501)
    lh = scenes._fm_lnh(a, l, r, np.full_like(r, np.pi / 2), 6.0)
    assert abs(r[np.argmax(lh)] - 12.0) < 0.02
    assert abs(r[np.argmin(np.abs(lh[:200]))] - 6.0) < 0.02

    def gBL(R):
        Sig, Del, A, s2 = scenes._kerr_bl(a, R, np.pi / 2)
        return -(1 - 2 * R / Sig), -2 * a * R * s2 / Sig, A * s2 / Sig

    for rr in [8.0, 12.0, 20.0]:
        Sig, Del, A, s2 = scenes._kerr_bl(a, rr, np.pi / 2)
        E = Sig * Sig * Del / (A * A * s2)
        U2 = 0.5 * (-1 + np.sqrt(1 + 4 * l * l * E))
        ut = np.sqrt(1 + U2) / np.sqrt(Sig * Del / A)
        up = ut * 2 * a * rr / A + np.sqrt(U2) / np.sqrt(A * s2 / Sig)
        Om = up / ut
        h = 1e-5
        f = lambda R: (lambda g: g[0] + 2 * Om * g[1] + Om * Om * g[2])(gBL(R))
        rhs = 0.5 * ut * ut * (f(rr + h) - f(rr - h)) / (2 * h)
        lhs = (scenes._fm_lnh(a, l, rr + h, np.pi / 2, 6.0) - scenes._fm_lnh(a, l, rr - h, np.pi / 2, 6.0)) / (2 * h)
        assert abs(lhs - rhs) < 1e-7
        g = gBL(rr)
        assert abs(g[0] * ut * ut + 2 * g[1] * ut * up + g[2] * up * up + 1) < 1e-12
        assert abs(ut * (g[1] * ut + g[2] * up) - l) < 1e-12


def test_torus_snapshots_shape_and_seed():
    f1, m = scenes.torus_snapshots(2, n1=32, n2=24, n_modes=64)
    f2, _ = scenes.torus_snapshots(2, n1=32, n2=24, n_modes=64)
    assert f1.shape == (2, 8, 24, 32) and f1.dtype == np.float32
    assert np.array_equal(f1, f2)
    assert np.all(f1[:, 0] > 0) and np.all(f1[:, 1] > 0)
    assert not np.array_equal(f1[0, 0], f1[1, 0])  # the noise is advected between snapshots
    assert np.array_equal(f1[0, 2:], f1[1, 2:])  # velocities and fields are stationary
