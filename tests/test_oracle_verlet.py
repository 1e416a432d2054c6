"""Pins of the oracle's velocity-Verlet integrator (sec. 2.2.2, Eqs. 16-19): its local error
against RK4 is third order in the step (so the dl^2/2 term and the averaged derivative are
both right), its global error in E, L, Q second order on the paper's test orbit, and the
re-evaluation lowers the error constant.  CPU only."""
import numpy as np
import pytest


def _state(ora, s, al, be, steps):
    """State after `steps` RK4 steps from the camera (away from the camera's flat region)."""
    x, k = ora.camera(s, al, be)
    for _ in range(steps):
        x, k = ora.rk4_step(s, x, k, ora.step_size(s, x, k))
    return x, k


@pytest.mark.parametrize("reeval", [False, True])
def test_local_error_third_order(ora, reeval):
    """One Verlet step from a state near the hole against RK4 over the same step: the
    difference shrinks by ~8 when the step halves (local error O(dl^3)); dropping the
    f dl^2 / 2 term of Eq. 16 or the average of Eq. 19 would leave O(dl^2)."""
    s = ora.scene(a=0.9, incl_deg=60.0)
    for al, be in [(4.0, 3.0), (-6.0, 1.0)]:
        x, k = _state(ora, s, al, be, 100)
        assert x[1] < 20.0
        f0 = ora.verlet_step(s, x, k, np.zeros(4), 0.0)[2]  # derivative at the point
        errs = []
        hs = [0.2, 0.1, 0.05, 0.025]
        for h in hs:
            xv, kv, _ = ora.verlet_step(s, x, k, f0, h, reeval)
            xr, kr = ora.rk4_step(s, x, k, h)
            errs.append(np.abs(np.concatenate([xv - xr, kv - kr])).max())
        slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
        assert 2.7 < slope < 3.3, (slope, errs)


def _L1_err(ora, eps, integ):
    s = ora.scene(a=0.998, incl_deg=90.0, eps=eps, r_cam=1000.0, integrator=integ)
    x, k = ora.camera(s, -3.22, 1.12)
    c0 = ora.constants(s, x, k)
    st, xf, kf, n = ora.geodesic(s, -3.22, 1.12)
    c1 = ora.constants(s, xf, kf)
    return np.abs(c1[:3] - c0[:3]), st


def test_global_error_second_order_and_reevaluation(ora):
    """Sec. 4.1's test orbit (a=0.998, i=90, alpha=-3.22, beta=1.12): the errors in E, L and
    Q of both Verlet variants converge at second order in eps (Q reaches its asymptotic
    rate below eps ~ 0.005), and the re-evaluated variant is the more accurate one."""
    epss = [0.005, 0.0025, 0.00125]
    res = {}
    for integ in (ora.VERLET, ora.VERLET_REEVAL):
        errs = []
        for e in epss:
            err, st = _L1_err(ora, e, integ)
            assert st in (0, 1)
            errs.append(err)
        errs = np.array(errs)
        for q in range(3):
            slope = np.polyfit(np.log(epss), np.log(errs[:, q]), 1)[0]
            assert 1.7 < slope < 2.3, (integ, q, slope, errs[:, q])
        res[integ] = errs
    assert np.exp(np.log(res[ora.VERLET_REEVAL]).mean()) < np.exp(np.log(res[ora.VERLET]).mean())


def test_verlet_trace_uses_one_start_derivative(ora):
    """A traced Verlet ray equals the same steps taken by hand with ora.verlet_step from the
    camera's derivative (the carried derivative is the one of the last evaluation)."""
    s = ora.scene(a=0.5, incl_deg=45.0, integrator=ora.VERLET_REEVAL)
    tr = ora.trace_ray(s, 5.0, 2.0, [230e9], max_trace=400)["trace"]
    x, k = ora.camera(s, 5.0, 2.0)
    f = ora.verlet_step(s, x, k, np.zeros(4), 0.0)[2]
    for t in tr[:200]:
        dl = ora.step_size(s, x, k)
        assert dl == t[8]
        x, k, f = ora.verlet_step(s, x, k, f, dl, True)
        assert np.array_equal(x, t[:4]) and np.array_equal(k, t[4:8])
