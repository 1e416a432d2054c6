"""FP64 CUDA path vs the FP64 CPU oracle: element-by-element parity (<= 1e-8 relative per
pixel, <= 1e-10 on the flux), identical step counts and termination codes, per-step trace
parity, full-size sampled parity and argument validation.  Needs a GPU."""
import math

import numpy as np
import pytest

from helpers import oracle_kwargs, rel_err
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu

PIX_TOL = 1e-8
FLUX_TOL = 1e-10


@pytest.fixture(scope="module")
def R():
    import torch

    assert torch.cuda.is_available()
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


def _ctx(R, cam, **over):
    c = dict(cam)
    c.update(over)
    ctx = R.Context(R.camera_desc(**c))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    return ctx


def _gpu_render(R, ctx, freqs, n_rows=None, row0=0):
    import torch

    ny = ctx.cam.ny if n_rows is None else n_rows
    steps = torch.zeros((ny, ctx.cam.nx), dtype=torch.int32, device="cuda")
    status = torch.zeros_like(steps)
    img, fl = ctx.render(freqs, row0=row0, n_rows=ny, steps=steps, status=status)
    torch.cuda.synchronize()
    return img.cpu().numpy(), fl, steps.cpu().numpy(), status.cpu().numpy()


def test_small_image_fp64_parity(R, ora):
    """64 x 64, a = 0.9, i = 60 deg, 230 GHz."""
    cam = scenes.SMALL
    ctx = _ctx(R, cam)
    img, fl, st, stat = _gpu_render(R, ctx, scenes.SMALL_FREQS)
    oimg, ost, ostat = ora.render(ora.scene(**oracle_kwargs(cam)), scenes.SMALL_FREQS)
    assert np.array_equal(stat, ostat)
    assert np.array_equal(st, ost)
    e = rel_err(img, oimg)
    assert e.max() <= PIX_TOL, e.max()
    assert abs(fl[0] / oimg.sum() - 1) <= FLUX_TOL
    assert abs(fl[0] - img.sum()) <= 1e-12 * abs(fl[0])


@pytest.mark.parametrize("spin", scenes.SPECTRAL_SPINS)
def test_ragged_multifrequency_fp64_parity(R, ora, spin):
    """8 log-spaced frequencies, a ragged 38 x 29 camera (not a multiple of the warp or
    block size) for each spin of the spectral workload."""
    cam = dict(scenes.SMALL, spin=spin, nx=38, ny=29)
    ctx = _ctx(R, cam)
    img, fl, st, stat = _gpu_render(R, ctx, scenes.SPECTRAL_FREQS)
    oimg, ost, ostat = ora.render(ora.scene(**oracle_kwargs(cam)), scenes.SPECTRAL_FREQS)
    assert np.array_equal(st, ost) and np.array_equal(stat, ostat)
    for f in range(len(scenes.SPECTRAL_FREQS)):
        e = rel_err(img[f], oimg[f])
        assert e.max() <= PIX_TOL, (f, e.max())
        assert abs(fl[f] / oimg[f].sum() - 1) <= FLUX_TOL


def test_polar_ray_degenerate_case(R, ora):
    """An odd camera width centred on alpha = 0 samples L = 0 exactly: that ray heads for
    the pole, which the step rule of Eqs. 20-23 approaches geometrically without crossing.
    Both implementations stop it (step cap or non-finite state) with a finite intensity,
    and every other pixel keeps parity."""
    cam = dict(scenes.SMALL, spin=0.5, nx=9, ny=6, max_steps=3000)
    ctx = _ctx(R, cam)
    img, fl, st, stat = _gpu_render(R, ctx, [1e11])
    oimg, ost, ostat = ora.render(ora.scene(**oracle_kwargs(cam)), [1e11])
    mid = cam["nx"] // 2
    assert np.all(np.isin(stat[:, mid], [R.RAY_TRUNCATED, R.RAY_ERROR, R.RAY_CAPTURED, R.RAY_ESCAPED]))
    assert np.all(np.isfinite(img))
    keep = np.ones(img.shape[1:], bool)
    keep[:, mid] = False
    assert np.array_equal(st[keep], ost[keep])
    assert rel_err(img[0][keep], oimg[0][keep]).max() <= PIX_TOL


def test_row_window_equals_full_image(R):
    cam = dict(scenes.SMALL, nx=32, ny=32)
    ctx = _ctx(R, cam)
    full, _, _, _ = _gpu_render(R, ctx, [1e11])
    part, _, _, _ = _gpu_render(R, ctx, [1e11], n_rows=7, row0=11)
    assert np.array_equal(part[0], full[0, 11:18])


def test_render_host_equals_device_render(R):
    """raptor_render_host (the end-to-end entry point: host image and flux) returns the device
    render's image and flux bit for bit, into a new array or into a given page-locked one;
    a wrong `out` is refused before anything runs."""
    import torch

    cam = dict(scenes.SMALL, nx=40, ny=24)
    freqs = [1e10, 230e9]
    ctx = _ctx(R, cam)
    img, fl = ctx.render(freqs)
    torch.cuda.synchronize()
    h, hfl = ctx.render_host(freqs)
    assert np.array_equal(h, img.cpu().numpy()) and np.array_equal(hfl, fl)
    out = R.pinned_host_array((2, 24, 40))
    out[:] = np.nan
    h2, hfl2 = ctx.render_host(freqs, out=out)
    assert h2 is out and np.array_equal(out, h) and np.array_equal(hfl2, fl)
    for bad in (np.zeros((2, 24, 41)), np.zeros((2, 24, 40), np.float32), np.zeros((40, 24, 2)).transpose(2, 1, 0)):
        with pytest.raises(ValueError):
            ctx.render_host(freqs, out=bad)


def test_single_pixel_and_many_frequencies(R, ora):
    """Degenerate sizes: one pixel; 20 frequencies (two frequency chunks of the kernel)."""
    cam = dict(scenes.SMALL, nx=1, ny=1, alpha_min=4.0, alpha_max=4.5, beta_min=1.0, beta_max=1.5)
    freqs = list(np.logspace(10, 13, 20))
    ctx = _ctx(R, cam)
    img, fl, st, stat = _gpu_render(R, ctx, freqs)
    oimg, ost, _ = ora.render(ora.scene(**oracle_kwargs(cam)), freqs)
    assert st[0, 0] == ost[0, 0]
    assert rel_err(img.ravel(), oimg.ravel()).max() <= PIX_TOL


@pytest.mark.parametrize("spin,incl", [(0.9, 5.0), (0.9, 90.0), (0.9, 150.0), (-0.7, 60.0), (0.998, 30.0)])
def test_inclinations_and_retrograde_spin(R, ora, spin, incl):
    """Camera geometry beyond the workloads' i = 60 deg: nearly face-on (the camera 5 deg
    from the axis), edge-on, below the equatorial plane (cos i < 0), a retrograde hole
    (a < 0: the analytic flow counter-rotates about the camera's axis, r_isco ~ 8.1 M) and a
    near-extremal prograde one; 40 x 36 pixels, two frequencies, every pixel and status
    against the oracle."""
    cam = dict(scenes.SMALL, spin=spin, incl_deg=incl, nx=40, ny=36)
    freqs = [86e9, 230e9]
    img, fl, st, stat = _gpu_render(R, _ctx(R, cam), freqs)
    oimg, ost, ostat = ora.render(ora.scene(**oracle_kwargs(cam)), freqs)
    assert np.array_equal(st, ost) and np.array_equal(stat, ostat)
    for f in range(len(freqs)):
        assert rel_err(img[f], oimg[f]).max() <= PIX_TOL, f
        assert abs(fl[f] / oimg[f].sum() - 1) <= FLUX_TOL, f


def test_polar_axis_rays_are_ill_conditioned(R, ora):
    """Rays of zero angular momentum (alpha = 0) pass the polar axis; the step rule's
    min(theta, pi - theta) factor shrinks the steps towards it and the turning point follows
    the rounding of L, so the transfer's samples there, and the pixel, follow tiny shifts of
    alpha.  On the FP64 path, which agrees with the oracle on such a pixel, a 1e-8 M shift of
    alpha at (0, 2.76 M) moves the pixel by more than the mixed paths' 1e-2 per-pixel bound,
    while the same shift at alpha = 0.0195 M (the 1024^2 headline's nearest column) and at
    0.1 M moves it by far less; the mixed-path tests exclude the strip |alpha| < 1e-3 M."""
    freqs = [6.158e10, 230e9]
    be = 2.7586206896551726

    def one(al):
        cam = dict(scenes.SMALL, nx=1, ny=1, alpha_min=al - 1e-9, alpha_max=al + 1e-9, beta_min=be - 1e-9,
                   beta_max=be + 1e-9)
        img, _, st, stat = _gpu_render(R, _ctx(R, cam), freqs)
        return cam, img[:, 0, 0], int(st[0, 0]), int(stat[0, 0])

    cam0, v0, n0, s0 = one(0.0)
    oimg, ost, ostat = ora.render(ora.scene(**oracle_kwargs(cam0)), freqs)
    assert n0 == ost[0, 0] and s0 == ostat[0, 0]
    assert np.abs(v0 / oimg[:, 0, 0] - 1).max() <= 1e-8
    _, v1, _, _ = one(1e-8)
    assert np.abs(v1 / v0 - 1).max() > 1e-2
    for al in (0.01953125, 0.1):
        _, w0, _, _ = one(al)
        _, w1, _, _ = one(al + 1e-8)
        assert np.abs(w1 / w0 - 1).max() < 1e-5, al


def test_trace_per_step_parity(R, ora):
    """Per-step states, step sizes, redshift factors, I and tau along selected rays."""
    cam = scenes.SMALL
    ctx = _ctx(R, cam)
    s = ora.scene(**oracle_kwargs(cam))
    for al, be in [(5.0, 3.0), (-3.0, 0.5), (0.31, -7.9), (15.0, 12.0)]:
        g = ctx.trace_ray(al, be, [230e9], max_rec=5000)
        o = ora.trace_ray(s, al, be, [230e9], max_trace=5000, t_cam=ctx.cam.t_delay)
        assert g["steps"] == o["steps"] and g["status"] == o["status"]
        tg, to = g["trace"], o["trace"]
        d = np.abs(tg - to)
        # positions/wave vectors/step sizes to 1e-10 of their magnitude (phi and t grow)
        assert np.all(d[:, :9] <= 1e-9 * np.maximum(np.abs(to[:, :9]), 1.0))
        # intensities along the ray, with the image tests' floor of 1e-12 of the final value
        floor = 1e-12 * abs(to[-1, 10])
        assert np.all(d[:, 10] <= PIX_TOL * np.maximum(np.abs(to[:, 10]), floor))
        assert math.isclose(g["I"][0], o["I"][0], rel_tol=PIX_TOL)


def test_headline_size_sampled_parity(R, ora):
    """The 1024 x 1024 headline image in the benchmark's launch configuration, checked on a
    seeded sample of pixels that the oracle traces one by one."""
    cam = scenes.HEADLINE
    ctx = _ctx(R, cam)
    img, fl, st, stat = _gpu_render(R, ctx, scenes.HEADLINE_FREQS)
    s = ora.scene(**oracle_kwargs(cam))
    al, be = R.pixel_centres(ctx.cam)
    pix = scenes.sample_pixels(cam["nx"], cam["ny"], 64, seed=1024)
    ref = img[0].max()
    Lcm = ora.length_unit_cm(cam["mass_msun"])
    D = cam["distance_pc"] * 3.0856775814913673e18
    pix_jy = (al[1] - al[0]) * (be[1] - be[0]) * Lcm**2 / D**2 / 1e-23
    for i, j in pix:
        o = ora.trace_ray(s, al[j], be[i], scenes.HEADLINE_FREQS)
        assert st[i, j] == o["steps"] and stat[i, j] == o["status"]
        ov = o["I"][0] * pix_jy
        assert abs(img[0, i, j] - ov) <= PIX_TOL * max(abs(ov), 1e-12 * ref)
    assert np.all(np.isfinite(img)) and np.all(img >= 0)
    assert abs(fl[0] - img.sum()) <= 1e-12 * fl[0]


def test_invalid_arguments_rejected(R):
    import torch

    with pytest.raises(R.RaptorError) as e:
        R.Context(R.camera_desc(spin=1.0))
    assert e.value.status == R.EINVAL
    with pytest.raises(R.RaptorError):
        R.Context(R.camera_desc(nx=0))
    ctx = R.Context(R.camera_desc(nx=8, ny=8))
    with pytest.raises(R.RaptorError) as e:
        ctx.render([230e9])
    assert e.value.status == R.ENOPLASMA
    ctx.load_plasma(R.plasma_desc())
    for bad in ([], [-1.0], [float("nan")], list(np.ones(65) * 1e11)):
        with pytest.raises(R.RaptorError) as e:
            ctx.render(bad if bad else np.zeros(0))
        assert e.value.status == R.EINVAL
    with pytest.raises(R.RaptorError):
        ctx.render([1e11], row0=5, n_rows=4)
    with pytest.raises(R.RaptorError) as e:
        ctx.load_plasma(R.plasma_desc(kind=R.PLASMA_GRID))
    assert e.value.status == R.EINVAL
    img, fl = ctx.render([1e11])
    torch.cuda.synchronize()
    assert np.isfinite(fl[0])


def test_step_cap_counts_truncated_rays(R):
    import torch

    ctx = _ctx(R, dict(scenes.SMALL, nx=8, ny=8, max_steps=20))
    steps = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    status = torch.zeros_like(steps)
    ctx.stats_reset()
    ctx.render([230e9], steps=steps, status=status)
    st = ctx.stats()
    assert np.all(steps.cpu().numpy() == 20)
    assert np.all(status.cpu().numpy() == R.RAY_TRUNCATED)
    assert st["truncated"] == 64 and st["rays"] == 64 and st["steps"] == 64 * 20


def test_invalid_arguments_of_the_options(R):
    """Argument checks of the schedule, profiling, disk and emissivity entry points (EINVAL,
    nothing launched) and that a context stays usable after them."""
    import torch

    ctx = R.Context(R.camera_desc(nx=8, ny=8))
    ctx.load_plasma(R.plasma_desc())
    bad_calls = [
        lambda: ctx.mixed_config(-1.0),
        lambda: ctx.mixed_config(0.5, [0]),
        lambda: ctx.mixed_config(0.5, None, -1),
        lambda: ctx.long_config(48),
        lambda: ctx.long_config(0, [0]),
        lambda: ctx.long_config(0, [1] * 8),
        lambda: ctx.disk_render(r_in=20.0, r_out=15.0),
        lambda: ctx.disk_render(max_cross=0),
        lambda: ctx.disk_render(n_bins=0),
        lambda: ctx.disk_render(x_range=(1.0, 0.5)),
        lambda: ctx.load_plasma(R.plasma_desc(theta_e_min=-1.0)),
        lambda: ctx.load_plasma(R.plasma_desc(theta_e_min=float("nan"))),
    ]
    for call in bad_calls:
        with pytest.raises(R.RaptorError) as e:
            call()
        assert e.value.status == R.EINVAL
    with pytest.raises(R.RaptorError) as e:
        R.Context(R.camera_desc(flags=0x40))
    assert e.value.status == R.EINVAL
    img, fl = ctx.render([1e11])
    torch.cuda.synchronize()
    assert np.isfinite(fl[0])
    d = ctx.disk_render()
    assert d["spectrum"].shape == (64,) and d["edges"].shape == (65,)
