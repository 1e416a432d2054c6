"""Pins of the oracle's adaptive step rule (sec. 2.2.2, Eqs. 20-23) and of the image's
scaling to Jy per pixel (sec. 4.2.2, the flux integration behind Table 3).  CPU only.

The step rule is pinned term by term on rays that isolate one term (the others vanish),
by the harmonic combination of three equal terms, by its polar symmetry and by the
far-field limit the analytic workload quotes (d lambda ~ 0.05 r).  The image scaling is
pinned by the total flux density of an optically thin-or-thick uniform ball in flat space,
whose closed form follows from the chord length through a sphere, and by how the image
scales with the mass and the distance."""
import math

import numpy as np
import pytest
from scipy import integrate

# CGS constants (CODATA 2018 / IAU 2015), typed here from their definitions
G_CGS, C_CGS, MSUN_G, PC_CM = 6.67430e-8, 2.99792458e10, 1.98841e33, 3.0856775814913673e18
EPS = 0.05


def _step(ora, s, r, th, k):
    return ora.step_size(s, np.array([0.0, r, th, 0.0]), np.asarray(k, float))


def test_step_radial_term(ora):
    """Eq. 20 read in x1 = ln r: a purely radial ray (k^theta = k^phi = 0) takes
    d lambda = eps r / |k^r|: the step is a fixed fraction eps of the e-folding length of
    r, independent of theta and of the sign of k^r."""
    s = ora.scene(eps=EPS)
    for r in (2.5, 6.0, 40.0, 1000.0):
        for kr in (-1.3, -0.2, 0.7, 2.0):
            for th in (0.3, 1.2, 2.9):
                dl = _step(ora, s, r, th, [1.0, kr, 0.0, 0.0])
                assert math.isclose(dl, EPS * r / abs(kr), rel_tol=1e-13), (r, kr, th)


def test_step_polar_term(ora):
    """Eq. 21 read in x2 = theta / pi: with only k^theta non-zero the step is
    eps min(x2, 1 - x2) / |dx2/dlambda| = eps min(theta, pi - theta) / |k^theta|, so a ray
    slows down geometrically as it approaches either pole, whatever its radius."""
    s = ora.scene(eps=EPS)
    for th in (1e-3, 0.1, 0.8, math.pi / 2, 2.5, math.pi - 1e-3):
        for kh in (-0.04, 0.01, 0.3):
            for r in (3.0, 50.0):
                dl = _step(ora, s, r, th, [1.0, 0.0, kh, 0.0])
                assert math.isclose(dl, EPS * min(th, math.pi - th) / abs(kh), rel_tol=1e-12), (th, kh, r)


def test_step_azimuthal_term(ora):
    """Eq. 22 with x3 = phi: with only k^phi non-zero, d lambda = eps / |k^phi| (a fixed
    fraction of a radian of azimuth per step)."""
    s = ora.scene(eps=EPS)
    for kp in (-0.5, 0.02, 3.0):
        for r, th in ((4.0, 1.0), (300.0, 0.2)):
            assert math.isclose(_step(ora, s, r, th, [1.0, 0.0, 0.0, kp]), EPS / abs(kp), rel_tol=1e-13)


def test_step_harmonic_combination(ora):
    """Eq. 23: the step is the harmonic combination 1/dl = 1/dl1 + 1/dl2 + 1/dl3 with equal
    weights.  With k^r = c r, k^theta = c theta (theta < pi/2) and k^phi = c, each term
    alone gives eps / c, so the combined step is eps / (3 c); two equal terms and a
    vanishing third give eps / (2 c)."""
    s = ora.scene(eps=EPS)
    for r, th, c in ((8.0, 0.7, 0.3), (2.2, 1.4, 1.7), (500.0, 0.05, 0.01)):
        dl = _step(ora, s, r, th, [1.0, c * r, c * th, c])
        assert math.isclose(dl, EPS / (3.0 * c), rel_tol=1e-12), (r, th, c)
        dl2 = _step(ora, s, r, th, [1.0, -c * r, 0.0, c])
        assert math.isclose(dl2, EPS / (2.0 * c), rel_tol=1e-12)
        # the polar term mirrored about the equator: theta -> pi - theta, k^theta -> -k^theta
        dlm = _step(ora, s, r, math.pi - th, [1.0, c * r, -c * th, c])
        assert math.isclose(dlm, dl, rel_tol=1e-12)


def test_step_far_field_limit_and_linear_rule(ora):
    """At the camera (r = 1000 M, k^r ~ 1 for the backward ray) the rule reduces to the
    workload's radius-scaled step d lambda ~ 0.05 r; the literal rule (flag) is exactly
    eps r for any wave vector."""
    s = ora.scene(eps=EPS)
    for al, be in ((3.0, 4.0), (-12.0, 0.5), (0.25, -18.0)):
        x, k = ora.camera(s, al, be)
        dl = ora.step_size(s, x, k)
        assert abs(dl / (EPS * x[1]) - 1.0) < 3e-2, (al, be, dl)
    lin = ora.scene(eps=EPS, step_rule=1)
    for r in (2.0, 30.0):
        assert _step(ora, lin, r, 1.0, [1.0, 0.3, 0.2, 0.1]) == pytest.approx(EPS * r, rel=1e-15)


def _ball_flux_jy(R, j, alpha, mass_msun, dist_pc):
    """Total flux density of a static uniform ball (radius R in units of GM/c^2, emission
    coefficient j, absorption alpha in cgs) seen from far away in flat space: each line of
    sight with impact parameter b crosses a chord 2 sqrt(R^2 - b^2), the formal solution of
    constant coefficients gives I(b) = (j/alpha)(1 - exp(-alpha chord)), and the flux
    density is the integral of I over the sky, 2 pi int I(b) b db / D^2, in Jy (1e-23 cgs)."""
    L = G_CGS * mass_msun * MSUN_G / C_CGS ** 2
    D = dist_pc * PC_CM

    def I(b):
        return j / alpha * -math.expm1(-alpha * 2.0 * math.sqrt(max(R * R - b * b, 0.0)) * L)

    val, _ = integrate.quad(lambda b: I(b) * b, 0.0, R, epsabs=0.0, epsrel=1e-12, limit=200)
    return 2.0 * math.pi * val * L * L / (D * D) / 1e-23


def _ball_scene(ora, n, R, jv, av, eps, mass=4.0e6, dist=7.88e3, half=None):
    half = R * 1.15 if half is None else half
    return ora.scene(m=0.0, a=0.0, plasma_kind=ora.KIND_BALL, ball_R=R, ball_j=jv, ball_alpha=av, eps=eps,
                     r_cam=200.0, r_esc=200.0, incl_deg=45.0, nx=n, ny=n, amin=-half, amax=half, bmin=-half,
                     bmax=half, mass_msun=mass, dist_pc=dist)


@pytest.mark.slow
def test_image_sum_is_flux_density_of_uniform_ball(ora):
    """Sec. 4.2.2 / Table 3: the image is Jy per pixel, I dalpha dbeta L^2 / D^2 / 1e-23, so
    its sum is the source's flux density.  For the flat-space uniform ball the sum must
    approach the closed form as the pixels and steps shrink (pixelisation of the limb and
    one misplaced step per boundary crossing are the only errors), both optically thin
    (alpha chord ~ 1e-3) and thick (~3)."""
    R = 6.0
    Lcm = G_CGS * 4.0e6 * MSUN_G / C_CGS ** 2
    for jv, av in ((1e-20, 1e-16), (3e-19, 2.5e-13)):
        exact = _ball_flux_jy(R, jv, av, 4.0e6, 7.88e3)
        errs = []
        for n, eps in ((24, 0.02), (48, 0.01), (96, 0.005)):
            img, _, status = ora.render(_ball_scene(ora, n, R, jv, av, eps), [1e11])
            assert np.all(status == ora.ESCAPED)
            errs.append(abs(img.sum() / exact - 1.0))
        assert errs[-1] < 1.5e-3, (av * 2 * R * Lcm, errs)
        assert errs[-1] < errs[0], errs


@pytest.mark.slow
def test_image_scaling_with_mass_and_distance(ora):
    """The image scales as L^2 / D^2 times the intensity: with the ball's coefficients fixed
    in cgs and its size fixed in units of GM/c^2, an optically thin ball's pixels scale as
    L^3 / D^2 (the chord is in cm, L ~ M).  Doubling M multiplies every pixel by 8, doubling
    D divides it by 4; an optically thick ball's pixels (I = j/alpha) scale as M^2."""
    R, eps, n = 6.0, 0.02, 24
    thin = _ball_scene(ora, n, R, 1e-20, 1e-22, eps)
    base, _, _ = ora.render(thin, [1e11])
    m2, _, _ = ora.render(_ball_scene(ora, n, R, 1e-20, 1e-22, eps, mass=8.0e6), [1e11])
    d2, _, _ = ora.render(_ball_scene(ora, n, R, 1e-20, 1e-22, eps, dist=2 * 7.88e3), [1e11])
    lit = base > 0
    assert lit.sum() > 100
    assert np.allclose(m2[lit] / base[lit], 8.0, rtol=1e-6)
    assert np.allclose(d2[lit] / base[lit], 0.25, rtol=1e-12)
    thick = _ball_scene(ora, n, R, 1e-17, 1e-8, eps)
    tb, _, _ = ora.render(thick, [1e11])
    tm, _, _ = ora.render(_ball_scene(ora, n, R, 1e-17, 1e-8, eps, mass=8.0e6), [1e11])
    lit = tb > 0
    assert np.allclose(tm[lit] / tb[lit], 4.0, rtol=1e-9)
    # thick pixels are the source function times the pixel's solid angle in Jy
    Lcm = G_CGS * 4.0e6 * MSUN_G / C_CGS ** 2
    D = 7.88e3 * PC_CM
    da = 2 * R * 1.15 / n
    assert np.allclose(tb[lit], 1e-17 / 1e-8 * da * da * Lcm * Lcm / (D * D) / 1e-23, rtol=1e-9)


def test_polar_axis_rays_are_ill_conditioned(ora):
    """The step rule near the polar axis (Eq. 21 as read): a ray of zero angular momentum
    (alpha = 0; L = -alpha sin i) passes within ~1e-6 rad of the axis, where the steps
    shrink like min(theta, pi - theta), and its transfer samples there follow shifts of
    alpha far below a pixel: at (0, 2.76 M) a 1e-8 M shift moves the intensity by more than
    1e-2, at alpha = 0.0195 M (the 1024^2 image's nearest column) and 0.1 M by less than
    1e-5.  This is why the mixed paths' per-pixel bound leaves out |alpha| < 1e-3 M and the
    learned path integrates |alpha| < 0.01 M from the camera."""
    from helpers import oracle_kwargs
    from paper_1801_10452_b300 import scenes

    s = ora.scene(**oracle_kwargs(dict(scenes.SMALL)))
    be, freqs = 2.7586206896551726, [6.158e10, 230e9]

    def trace(al):
        return ora.trace_ray(s, al, be, freqs, max_trace=5000)

    o0, o1 = trace(0.0), trace(1e-8)
    th = o0["trace"][:, 2]
    assert np.minimum(th, np.pi - th).min() < 1e-5
    assert np.abs(o1["I"] / o0["I"] - 1).max() > 1e-2
    for al in (0.01953125, 0.1):
        a, b = trace(al), trace(al + 1e-8)
        assert np.abs(b["I"] / a["I"] - 1).max() < 1e-5, al
