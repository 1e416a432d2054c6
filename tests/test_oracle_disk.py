"""Pins of the oracle's thin-disk line emitter (sec. 4.2.1) against closed forms: the
redshift of an equatorial circular Keplerian emitter in terms of the camera's conserved
quantities (Bardeen, Press & Teukolsky), the crossing point against bisection, the disk's
radial extent, and the bookkeeping of the line spectrum.  CPU only."""
import math

import numpy as np
import pytest


def _ut_omega(a, r):
    """u^t and Omega of a prograde circular equatorial orbit (BPT 1972; a < 0: retrograde
    relative to the hole)."""
    ut = (r**1.5 + a) / (r**0.75 * math.sqrt(r**1.5 - 3.0 * r**0.5 + 2.0 * a))
    return ut, 1.0 / (r**1.5 + a)


def _hits(ora, s, n, seed, half=15.0):
    rng = np.random.default_rng(seed)
    out = []
    for al, be in rng.uniform(-half, half, (n, 2)):
        d = ora.disk_ray(s, al, be)
        if d["status"] == ora.DISK_HIT:
            out.append((al, be, d))
    return out


@pytest.mark.parametrize("a,incl", [(0.5, 30.0), (-0.9, 60.0), (0.99, 85.0), (0.0, 30.0), (-0.5, 45.0)])
def test_redshift_matches_keplerian_closed_form(ora, a, incl):
    """g = k.u at the hit equals u^t (1 - Omega L) with L = -alpha sin i the camera's
    conserved angular momentum (k_t = -1) and u^t, Omega of the circular orbit at the hit's
    radius.  The integrated k_t, k_phi drift like eps^4: at eps = 0.01 the two agree to 1e-8;
    the same rays at eps = 0.05 differ by ~1e-6, consistent with fourth order."""
    fine = ora.scene(a=a, incl_deg=incl, eps=0.01)
    hits = _hits(ora, fine, 60, seed=int(100 * (a + 2) + incl))
    assert len(hits) >= 5
    sin_i = math.sin(math.radians(incl))
    for al, be, d in hits:
        ut, om = _ut_omega(a, d["r"])
        cf = ut * (1.0 - om * (-al * sin_i))
        assert abs(d["g"] / cf - 1.0) <= 1e-8, (al, be, d["g"], cf)
        assert abs(d["ratio"] * d["g"] - 1.0) <= 1e-15
        assert abs(d["theta"] - 0.5 * math.pi) <= 1e-12
        assert d["I"] == pytest.approx(d["ratio"] ** 4 * d["r"] ** -2.0, rel=1e-14)
    coarse = ora.scene(a=a, incl_deg=incl, eps=0.05)
    worst = 0.0
    for al, be, _ in hits[:5]:
        d = ora.disk_ray(coarse, al, be)
        if d["status"] == ora.DISK_HIT:
            ut, om = _ut_omega(a, d["r"])
            worst = max(worst, abs(d["g"] / (ut * (1.0 - om * (-al * sin_i))) - 1.0))
    assert 1e-8 < worst < 1e-4


def test_crossing_point_against_bisection(ora):
    """The Newton-refined crossing equals the point found by bisection on the length of one
    RK4 step from the state before the crossing step (the oracle's own RK4, traced)."""
    s = ora.scene(a=0.7, incl_deg=50.0)
    for al, be in [(6.0, 2.0), (-9.0, 4.0), (2.0, -7.5), (11.0, -1.0)]:
        d = ora.disk_ray(s, al, be)
        assert d["status"] == ora.DISK_HIT and d["order"] == 1
        tr = ora.trace_ray(s, al, be, [230e9], max_trace=2000)["trace"]
        x0, k0 = ora.camera(s, al, be)
        states = [(x0, k0)] + [(t[:4], t[4:8]) for t in tr]
        for n in range(1, len(states)):
            if (states[n - 1][0][2] - 0.5 * math.pi) * (states[n][0][2] - 0.5 * math.pi) <= 0.0:
                break
        xs, ks = states[n - 1]
        dl = tr[n - 1][8]
        lo, hi = 0.0, dl
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            xm, km = ora.rk4_step(s, xs.copy(), ks.copy(), mid)
            if (xm[2] - 0.5 * math.pi) * (xs[2] - 0.5 * math.pi) > 0.0:
                lo = mid
            else:
                hi = mid
        xm, _ = ora.rk4_step(s, xs.copy(), ks.copy(), 0.5 * (lo + hi))
        assert abs(xm[1] - d["r"]) <= 1e-10 * d["r"], (al, be)


@pytest.mark.parametrize("a", [0.99, 0.0, -0.99])
def test_hits_lie_on_the_disk(ora, a):
    """Every hit lies between the ISCO (BPT) and 15 M; with an explicit inner radius the
    hits respect it; rays through the hole's shadow are captured, not hit."""
    s = ora.scene(a=a, incl_deg=60.0)
    ri = ora.r_isco(a)
    for _, _, d in _hits(ora, s, 40, seed=7):
        assert ri - 1e-12 <= d["r"] <= 15.0 + 1e-12
        assert d["order"] >= 1
    for _, _, d in [(0, 0, ora.disk_ray(s, al, be, r_in=10.0)) for al, be in [(3.0, 3.0), (-12.0, 1.0)]]:
        assert d["status"] != ora.DISK_HIT or 10.0 <= d["r"] <= 15.0
    assert ora.disk_ray(s, 0.05, 0.05)["status"] == ora.CAPTURED


def test_face_on_schwarzschild_line_is_pure_gravitational(ora):
    """a = 0 seen nearly face-on: L ~ 0 for every ray, so E_obs/E_em = sqrt(1 - 3/r) at the
    hit (the transverse Doppler and gravitational shifts of a circular orbit) and the
    first-order line lies within [sqrt(1 - 3/6), sqrt(1 - 3/15)]."""
    s = ora.scene(a=0.0, incl_deg=1e-3, nx=24, ny=24, amin=-16.0, amax=16.0, bmin=-16.0, bmax=16.0)
    ratio, inten, order, status, _ = ora.disk_render(s)
    hit = order == 1
    assert hit.sum() > 100
    assert (ratio[hit] >= math.sqrt(0.5) - 1e-5).all() and (ratio[hit] <= math.sqrt(0.8) + 1e-5).all()
    al = -16.0 + (np.arange(24) + 0.5) * (32.0 / 24)
    d = ora.disk_ray(s, al[5], al[9])
    assert d["ratio"] == pytest.approx(math.sqrt(1.0 - 3.0 / d["r"]), rel=1e-5)


def test_line_profile_bookkeeping(ora):
    """The spectrum sums I * pixel area over first-order hits into bins [e_b, e_{b+1});
    its total equals the weight of the hits inside the range, a value on an edge goes to the
    upper bin, and higher-order hits (present at high inclination) are left out."""
    s = ora.scene(a=0.9, incl_deg=80.0, nx=32, ny=32, amin=-16.0, amax=16.0, bmin=-16.0, bmax=16.0)
    ratio, inten, order, status, _ = ora.disk_render(s)
    assert (order >= 2).any() and (order == 1).sum() > (order >= 2).sum()
    rng = (0.2, 1.6, 56)
    h = ora.line_profile(ratio, inten, order, *rng, 1.0)
    sel = (order == 1) & (ratio >= 0.2) & (ratio < 1.6)
    assert h.sum() == pytest.approx(inten[sel].sum(), rel=1e-12)
    h_all = ora.line_profile(ratio, inten, order, *rng, 1.0, profile_order=0)
    assert h_all.sum() > h.sum()
    edge = 0.2 + 10 * (1.4 / 56)
    one = np.ones((1, 1))
    assert ora.line_profile(one * 0.5, one, one.astype(int), 0.0, 1.0, 4, 1.0)[2] == 1.0
    assert ora.line_profile(one * 1.0, one, one.astype(int), 0.0, 1.0, 4, 1.0).sum() == 0.0
    assert ora.line_profile(one * edge, one, one.astype(int), *rng, 1.0).sum() == 1.0


def _schwarzschild_crossings(alpha, beta, incl_deg, r_cam, r_stop, r_esc, max_n=4):
    """Equatorial crossings of a Schwarzschild ray by quadrature of the orbit equation.  The
    orbit lies in the plane of the camera direction o = (sin i, 0, cos i) and the impact
    vector (alpha e_alpha + beta e_beta, e_beta = (-cos i, 0, sin i)); its angle from o is
    psi(u) = int du / sqrt(F(u)), F = 1/b^2 - u^2 + 2 u^3 (u = 1/r, b^2 = alpha^2 + beta^2),
    and the affine length lambda(u) = int du / (u^2 b sqrt(F)) (E = 1).  The plane z = 0 is
    met at psi_n = atan2(cos i, -beta sin i / b) + (n - 1) pi.  Near the turning point
    u_p (F = 2 (u - u1)(u - u_p)(u - u3)) the substitution u = u_p - s^2 removes the
    inverse square root.  Returns (r_n, lambda_n) of the crossings before capture or escape."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    b = math.hypot(alpha, beta)
    si, ci = math.sin(math.radians(incl_deg)), math.cos(math.radians(incl_deg))
    psi1 = math.atan2(ci, -beta * si / b)
    u0 = 1.0 / r_cam
    F = lambda u: 1.0 / b**2 - u * u + 2.0 * u**3
    roots = np.sort(np.roots([2.0, -1.0, 0.0, 1.0 / b**2]).real) if b > 3.0 * math.sqrt(3.0) else None
    opts = dict(epsabs=0.0, epsrel=1e-13, limit=200)
    if roots is None:
        # captured: psi and lambda grow monotonically to the stop radius
        u_end = 1.0 / r_stop
        psi = lambda u: quad(lambda v: 1.0 / math.sqrt(F(v)), u0, u, **opts)[0]
        lam = lambda u: quad(lambda v: 1.0 / (v * v * b * math.sqrt(F(v))), u0, u, **opts)[0]
        out = []
        for n in range(max_n):
            target = psi1 + n * math.pi
            if psi(u_end) < target:
                break
            u = brentq(lambda v: psi(v) - target, u0, u_end, xtol=1e-15, rtol=1e-15)
            out.append((1.0 / u, lam(u)))
        return out
    u1, up, u3 = roots

    def smooth(s, w):  # integrand in s for psi (w = 0) or lambda (w = 1), u = up - s^2
        u = up - s * s
        g = 2.0 / math.sqrt(2.0 * (u - u1) * (u3 - u))
        return g if w == 0 else g / (u * u * b)

    s0 = math.sqrt(up - u0)
    psi_in = lambda u: quad(smooth, math.sqrt(up - u), s0, args=(0,), **opts)[0]
    lam_in = lambda u: quad(smooth, math.sqrt(up - u), s0, args=(1,), **opts)[0]
    psi_p, lam_p = psi_in(up), lam_in(up)
    u_esc = 1.0 / r_esc
    out = []
    for n in range(max_n):
        target = psi1 + n * math.pi
        if target <= psi_p:  # inbound leg
            u = brentq(lambda v: psi_in(v) - target, u0, up, xtol=1e-16, rtol=1e-15)
            out.append((1.0 / u, lam_in(u)))
        else:  # outbound leg: psi = 2 psi_p - psi_in(u)
            rest = 2.0 * psi_p - target
            if rest < psi_in(u_esc):
                break
            u = brentq(lambda v: psi_in(v) - rest, u_esc, up, xtol=1e-16, rtol=1e-15)
            out.append((1.0 / u, 2.0 * lam_p - lam_in(u)))
    return out


@pytest.mark.parametrize("incl", [30.0, 60.0, 85.0])
def test_crossings_match_schwarzschild_quadrature(ora, incl):
    """a = 0: the oracle's ordered equatorial crossings (radius and affine length from the
    camera) equal the quadrature of the orbit equation, for escaping rays with one and two
    crossings (inbound and outbound legs) and a captured ray; the counts agree, and the
    difference shrinks like eps^4 (16x from eps = 0.02 to 0.01)."""
    rays = [(6.0, 2.0), (-7.0, -3.0), (5.25, 0.5), (-5.3, 0.4), (2.0, 1.0), (0.5, -3.5), (11.0, 4.0)]
    worst = {}
    for eps in (0.02, 0.01):
        s = ora.scene(a=0.0, incl_deg=incl, eps=eps, r_cam=1000.0)
        r_stop = 1.01 * 2.0
        w = 0.0
        for al, be in rays:
            c = ora.disk_crossings(s, al, be, 4)
            ref = _schwarzschild_crossings(al, be, incl, 1000.0, r_stop, 1000.0)
            assert len(c["r"]) == len(ref), (al, be, c, ref)
            for n, (rq, lq) in enumerate(ref):
                w = max(w, abs(c["r"][n] / rq - 1.0), abs(c["lam"][n] - lq) / rq)
            assert c["fate"] == (ora.CAPTURED if math.hypot(al, be) < 3.0 * math.sqrt(3.0) else ora.ESCAPED)
        worst[eps] = w
    assert worst[0.01] < 5e-7, worst
    assert worst[0.02] / worst[0.01] > 8.0, worst


def test_crossings_agree_with_the_disk_ray(ora):
    """The first crossing inside [r_in, r_out] of the crossing list is the disk ray's hit (same
    radius, same order); a ray whose crossings all miss the disk is a miss."""
    s = ora.scene(a=0.9, incl_deg=75.0)
    rng = np.random.default_rng(3)
    n_hit = 0
    for al, be in rng.uniform(-12.0, 12.0, (40, 2)):
        c = ora.disk_crossings(s, al, be, 10)
        d = ora.disk_ray(s, al, be)
        ri = ora.r_isco(0.9)
        inside = [n for n, r in enumerate(c["r"]) if ri <= r <= 15.0]
        if d["status"] == ora.DISK_HIT:
            n_hit += 1
            assert inside and inside[0] + 1 == d["order"] and c["r"][inside[0]] == d["r"]
        else:
            assert not inside
    assert n_hit >= 10
