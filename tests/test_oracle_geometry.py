"""Pins of the oracle's spacetime and geodesic machinery against closed forms and the
invariants the paper uses (sec. 2, sec. 4.1, App. A).  CPU only."""
import math

import numpy as np
import pytest

RNG = np.random.default_rng(20180131)


def _pts(n=20):
    r = RNG.uniform(1.6, 50.0, n)
    th = RNG.uniform(0.05, math.pi - 0.05, n)
    return zip(r, th)


@pytest.mark.parametrize("coords", [0, 1])
@pytest.mark.parametrize("a", [0.0, 0.5, 0.9375, -0.7])
def test_inverse_metric_textbook(ora, coords, a):
    """g^{mu nu} of Kerr in KS and BL (textbook closed forms) and det g = -Sigma^2 sin^2."""
    s = ora.scene(a=a, coords=coords)
    for r, th in _pts():
        g, gi = ora.metric(s, r, th)
        Sig = r * r + a * a * math.cos(th) ** 2
        Del = r * r - 2 * r + a * a
        s2 = math.sin(th) ** 2
        assert np.allclose(g @ gi, np.eye(4), atol=1e-12)
        assert np.isclose(np.linalg.det(g), -Sig**2 * s2, rtol=1e-10)
        if coords == 0:
            exp = np.zeros((4, 4))
            exp[0, 0] = -(1 + 2 * r / Sig)
            exp[0, 1] = exp[1, 0] = 2 * r / Sig
            exp[1, 1] = Del / Sig
            exp[1, 3] = exp[3, 1] = a / Sig
            exp[2, 2] = 1 / Sig
            exp[3, 3] = 1 / (Sig * s2)
        else:
            A = (r * r + a * a) ** 2 - a * a * Del * s2
            exp = np.zeros((4, 4))
            exp[0, 0] = -A / (Sig * Del)
            exp[0, 3] = exp[3, 0] = -2 * a * r / (Sig * Del)
            exp[1, 1] = Del / Sig
            exp[2, 2] = 1 / Sig
            exp[3, 3] = (Del - a * a * s2) / (Sig * Del * s2)
        assert np.allclose(gi, exp, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("a", [0.0, 0.6, 0.998])
def test_ks_metric_is_transformed_bl(ora, a):
    """App. A.1: dt~ = dt + 2r/Delta dr, dphi~ = dphi + a/Delta dr; so
    g_KS = Lambda^T g_BL Lambda with Lambda = d x_BL / d x_KS."""
    ks, bl = ora.scene(a=a, coords=0), ora.scene(a=a, coords=1)
    for r, th in _pts():
        if r * r - 2 * r + a * a <= 1e-3:
            continue
        gk, _ = ora.metric(ks, r, th)
        gb, _ = ora.metric(bl, r, th)
        Del = r * r - 2 * r + a * a
        Lam = np.eye(4)
        Lam[0, 1] = -2 * r / Del
        Lam[3, 1] = -a / Del
        assert np.allclose(Lam.T @ gb @ Lam, gk, rtol=1e-10, atol=1e-10)
        # the vector transform of the oracle is the inverse of Lam
        v = RNG.normal(size=4)
        vk = ora.vec_bl_to_ks(ks, r, v)
        assert np.allclose(Lam @ vk, v, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("a", [0.3, 0.9])
def test_ks_position_transform_matches_vector_transform(ora, a):
    """App. A.1: d t~/dr = 2r/Delta and d phi~/dr = a/Delta (central differences of the
    position map)."""
    s = ora.scene(a=a)
    for r in [2.5, 4.0, 10.0, 100.0]:
        h = 1e-5 * r
        xp = ora.pos_bl_to_ks(s, [0.0, r + h, 1.0, 0.0])
        xm = ora.pos_bl_to_ks(s, [0.0, r - h, 1.0, 0.0])
        Del = r * r - 2 * r + a * a
        assert math.isclose((xp[0] - xm[0]) / (2 * h), 2 * r / Del, rel_tol=1e-7)
        assert math.isclose((xp[3] - xm[3]) / (2 * h), a / Del, rel_tol=1e-7)


@pytest.mark.parametrize("coords", [0, 1])
def test_metric_derivatives_finite_difference(ora, coords):
    s = ora.scene(a=0.9, coords=coords)
    for r, th in _pts(10):
        dg = ora.dmetric(s, r, th)
        for l, (dr, dth) in ((1, (1e-6 * r, 0)), (2, (0, 1e-6))):
            gp, _ = ora.metric(s, r + dr, th + dth)
            gm, _ = ora.metric(s, r - dr, th - dth)
            fd = (gp - gm) / (2 * (dr + dth))
            assert np.allclose(dg[l], fd, rtol=1e-6, atol=1e-8 * max(1, np.abs(gp).max()))
        assert np.all(dg[0] == 0) and np.all(dg[3] == 0)


def test_connection_schwarzschild_textbook(ora):
    """Eq. 2 reproduces the textbook Schwarzschild Christoffel symbols (BL, M=1)."""
    s = ora.scene(a=0.0, coords=1)
    for r, th in _pts(10):
        if r < 2.2:
            continue
        G = ora.connection(s, r, th)
        f = 1 - 2 / r
        assert math.isclose(G[1, 0, 0], f / r**2, rel_tol=1e-12)
        assert math.isclose(G[0, 0, 1], 1 / (r * r * f), rel_tol=1e-12)
        assert math.isclose(G[1, 1, 1], -1 / (r * r * f), rel_tol=1e-12)
        assert math.isclose(G[1, 2, 2], -(r - 2), rel_tol=1e-12)
        assert math.isclose(G[1, 3, 3], -(r - 2) * math.sin(th) ** 2, rel_tol=1e-12)
        assert math.isclose(G[2, 1, 2], 1 / r, rel_tol=1e-12)
        assert math.isclose(G[3, 1, 3], 1 / r, rel_tol=1e-12)
        assert math.isclose(G[2, 3, 3], -math.sin(th) * math.cos(th), rel_tol=1e-12)
        assert math.isclose(G[3, 2, 3], math.cos(th) / math.sin(th), rel_tol=1e-12)
        assert np.allclose(G, np.transpose(G, (0, 2, 1)), atol=0)


@pytest.mark.parametrize("coords", [0, 1])
def test_connection_symmetric_and_fd(ora, coords):
    """Gamma symmetric in the lower indices; equals Eq. 2 built from finite differences."""
    s = ora.scene(a=0.9, coords=coords)
    for r, th in _pts(5):
        G = ora.connection(s, r, th)
        assert np.allclose(G, np.transpose(G, (0, 2, 1)), rtol=0, atol=1e-15 * np.abs(G).max())
        g, gi = ora.metric(s, r, th)
        d = np.zeros((4, 4, 4))
        for l, (dr, dth) in ((1, (1e-6 * r, 0)), (2, (0, 1e-6))):
            gp, _ = ora.metric(s, r + dr, th + dth)
            gm, _ = ora.metric(s, r - dr, th - dth)
            d[l] = (gp - gm) / (2 * (dr + dth))
        Gfd = 0.5 * (np.einsum("ar,mnr->amn", gi, d) + np.einsum("ar,nmr->amn", gi, d) - np.einsum("ar,rmn->amn", gi, d))
        assert np.allclose(G, Gfd, rtol=1e-5, atol=1e-7 * np.abs(G).max())


@pytest.mark.parametrize("coords", [0, 1])
@pytest.mark.parametrize("a,incl", [(0.9, 60.0), (0.0, 30.0), (0.998, 90.0), (-0.5, 17.0)])
def test_camera_null_and_constants(ora, coords, a, incl):
    """Sec. 2.3: the camera wave vector is null (Eq. 4) and carries E=1,
    L = -alpha sin i, Q = beta^2 + cos^2 i (alpha^2 - a^2) (Eq. 39 at the camera)."""
    s = ora.scene(a=a, coords=coords, incl_deg=incl)
    for al, be in [(5.0, 3.0), (-3.22, 1.12), (0.3, -7.0), (-15.0, -0.2), (19.0, 19.0)]:
        x, k = ora.camera(s, al, be)
        E, L, Q, kk = ora.constants(s, x, k)
        i = math.radians(incl)
        assert math.isclose(E, 1.0, rel_tol=1e-13)
        assert math.isclose(L, -al * math.sin(i), rel_tol=1e-12, abs_tol=1e-13)
        assert math.isclose(Q, be * be + math.cos(i) ** 2 * (al * al - a * a), rel_tol=1e-10, abs_tol=1e-10)
        assert abs(kk) < 1e-12
        assert k[1] < 0  # the backward ray heads inward
        assert (k[0] < 0)  # and into the past


def test_r_isco_closed_form_limits(ora):
    assert math.isclose(ora.r_isco(0.0), 6.0, rel_tol=1e-14)
    assert math.isclose(ora.r_isco(1.0), 1.0, rel_tol=1e-12)
    assert math.isclose(ora.r_isco(-1.0), 9.0, rel_tol=1e-12)
    r = [ora.r_isco(a) for a in np.linspace(-0.99, 0.99, 21)]
    assert np.all(np.diff(r) < 0)


def _rhs_kk_norm(ora, s, x, u):
    G = ora.connection(s, x[1], x[2])
    return np.einsum("amn,m,n->a", G, u, u)


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9375])
def test_analytic_plasma_velocity(ora, a):
    """Keplerian flow (r >= r_isco) and free fall (r < r_isco): u.u = -1 in KS; the
    equatorial Keplerian orbit is a geodesic (Gamma^r u u = 0); free fall has u_t = -1,
    u_phi = 0; b . u = 0 and |b| = B."""
    s = ora.scene(a=a)
    ri = ora.r_isco(a)
    rh = ora.horizon(s)
    for r in [1.02 * rh, 0.5 * (rh + ri), ri * 1.0001, 8.0, 30.0, 500.0]:
        for th in [0.3, 1.0, math.pi / 2, 2.5]:
            x = np.array([0.0, r, th, 0.0])
            ok, ne, te, B, u, b = ora.plasma(s, x)
            assert ok == 1
            g, _ = ora.metric(s, r, th)
            assert math.isclose(u @ g @ u, -1.0, rel_tol=1e-11)
            assert abs(b @ g @ u) < 1e-10 * B
            assert math.isclose(math.sqrt(b @ g @ b), B, rel_tol=1e-11)
            assert math.isclose(ne, 1e6 * r**-1.5, rel_tol=1e-14)
            ucov = g @ u
            if r < ri:
                assert math.isclose(ucov[0], -1.0, rel_tol=1e-10)
                assert abs(ucov[3]) < 1e-10
                assert u[2] == 0
            elif th == math.pi / 2:
                acc = _rhs_kk_norm(ora, s, x, u)
                assert abs(acc[1]) < 1e-11 * max(1.0, abs(u[0]) ** 2)


def test_static_plasma_redshift_is_gravitational(ora):
    """a = 0 static emitter: nu_fluid / nu_obs = 1/sqrt(1 - 2/r) at every sample of every ray
    (to the integrator's truncation error, which grows where the backward ray nears the
    horizon and its wave vector diverges in KS coordinates)."""
    s = ora.scene(a=0.0, plasma_kind=ora.KIND_STATIC_ISO, eps=0.02)
    for al, be in [(6.0, 1.0), (-2.0, 2.0), (12.0, -9.0)]:
        tr = ora.trace_ray(s, al, be, [230e9], max_trace=5000)["trace"]
        r, gr = tr[:, 1], tr[:, 9]
        m = (gr > 0) & (r > 2.5)
        assert m.sum() > 50
        assert np.allclose(gr[m], 1 / np.sqrt(1 - 2 / r[m]), rtol=1e-7)


def _L1_err(ora, eps):
    s = ora.scene(a=0.998, incl_deg=90.0, eps=eps, r_cam=1000.0)
    x, k = ora.camera(s, -3.22, 1.12)
    c0 = ora.constants(s, x, k)
    st, xf, kf, n = ora.geodesic(s, -3.22, 1.12)
    c1 = ora.constants(s, xf, kf)
    return np.abs(c1[:3] - c0[:3]), n, st


def test_rk4_conserves_constants_fourth_order(ora):
    """Sec. 4.1 / Fig. 6: along the orbit (a=0.998, i=90, alpha=-3.22, beta=1.12) the
    errors in E, L and Q converge at fourth order in the step for RK4."""
    epss = [0.08, 0.04, 0.02, 0.01]
    errs = []
    for e in epss:
        err, n, st = _L1_err(ora, e)
        assert st in (0, 1)
        errs.append(err)
    errs = np.array(errs)
    for q in range(3):
        slope = np.polyfit(np.log(epss), np.log(errs[:, q]), 1)[0]
        assert 3.3 < slope < 4.7, (q, slope, errs[:, q])
    assert errs[-1].max() < 1e-6


@pytest.mark.parametrize("orbit", [(0.998, 90.0, -2.1109, 0.0), (0.998, 60.0, -0.001, 4.752)])
def test_difficult_orbits_conserve_constants(ora, orbit):
    """Table 1's two difficult geodesics: invariants conserved and the null condition kept."""
    a, inc, al, be = orbit
    s = ora.scene(a=a, incl_deg=inc, eps=0.01)
    x, k = ora.camera(s, al, be)
    c0 = ora.constants(s, x, k)
    st, xf, kf, n = ora.geodesic(s, al, be)
    c1 = ora.constants(s, xf, kf)
    assert st in (0, 1)
    assert abs(c1[0] - c0[0]) < 1e-7 and abs(c1[1] - c0[1]) < 1e-6 and abs(c1[2] - c0[2]) < 1e-5
    assert abs(c1[3]) < 1e-6 * max(1.0, kf[0] ** 2)


def test_schwarzschild_shadow_radius(ora):
    """a = 0: rays with impact parameter b < 3 sqrt(3) M are captured, b > 3 sqrt(3) escape;
    bisection on b converges to 3 sqrt(3) = 5.19615..."""
    s = ora.scene(a=0.0, incl_deg=60.0, eps=0.01, r_cam=1000.0)
    lo, hi = 4.5, 6.0
    for _ in range(22):
        mid = 0.5 * (lo + hi)
        st, *_ = ora.geodesic(s, mid * math.cos(0.7), mid * math.sin(0.7))
        if st == 1:
            lo = mid
        else:
            hi = mid
    # r_cam = 1000 is finite: the impact parameter at infinity differs by O(M/r_cam)^2
    assert abs(0.5 * (lo + hi) - 3 * math.sqrt(3)) < 2e-3


def _bardeen_curve(a, inc, n=24):
    """Critical curve on the observer's sky (Bardeen 1973): photon-orbit radius r gives
    xi = L/E and eta = Q/E^2; alpha = -xi / sin i, beta = +-sqrt(eta + a^2 cos^2 i - xi^2 cot^2 i)."""
    rp = 2 * (1 + math.cos(2 / 3 * math.acos(-a)))
    rm = 2 * (1 + math.cos(2 / 3 * math.acos(a)))
    out = []
    for r in np.linspace(rp, rm, 400):
        xi = -(r**3 - 3 * r**2 + a * a * r + a * a) / (a * (r - 1))
        eta = r**3 * (4 * a * a - r * (r - 3) ** 2) / (a * a * (r - 1) ** 2)
        ci, si = math.cos(math.radians(inc)), math.sin(math.radians(inc))
        b2 = eta + a * a * ci * ci - xi * xi * ci * ci / (si * si)
        if b2 >= 0:
            out.append((-xi / si, math.sqrt(b2)))
    out = np.array(out)
    idx = np.linspace(0, len(out) - 1, n).astype(int)
    return out[idx]


def test_kerr_critical_curve_classification(ora):
    """a = 0.9, i = 60 deg: sky points 0.1 M inside Bardeen's critical curve are captured,
    0.1 M outside escape."""
    a, inc = 0.9, 60.0
    s = ora.scene(a=a, incl_deg=inc, eps=0.02)
    pts = _bardeen_curve(a, inc)
    c = pts.mean(axis=0) * np.array([1.0, 0.0])
    for al, be in pts:
        d = np.array([al, be]) - c
        d /= np.linalg.norm(d)
        st_in, *_ = ora.geodesic(s, al - 0.1 * d[0], be - 0.1 * d[1])
        st_out, *_ = ora.geodesic(s, al + 0.1 * d[0], be + 0.1 * d[1])
        assert st_in == 1 and st_out == 0, (al, be)


def test_camera_k_theta_reading(ora):
    """Eq. 28 at the camera (theta = i): Q - L^2 cot^2 + a^2 cos^2 = beta^2, so
    k_theta = beta.  Checked in extended precision against the printed form."""
    import numpy as np

    for a, inc in [(0.9, 60.0), (0.0, 17.0), (0.998, 85.0)]:
        s = ora.scene(a=a, incl_deg=inc, coords=1)
        for al, be in [(7.3, 0.0), (-3.1, 2.2), (15.0, -0.01)]:
            i = np.longdouble(math.radians(inc))
            A, Bt = np.longdouble(al), np.longdouble(be)
            L = -A * np.sin(i)
            Q = Bt * Bt + np.cos(i) ** 2 * (A * A - np.longdouble(a) ** 2)
            printed = Q - L * L * (np.cos(i) / np.sin(i)) ** 2 + np.longdouble(a) ** 2 * np.cos(i) ** 2
            assert abs(float(printed) - be * be) < 1e-15 * max(1.0, al * al)
            x, k = ora.camera(s, al, be)
            g, _ = ora.metric(s, x[1], x[2])
            kc = g @ (-k)
            assert kc[2] == be
