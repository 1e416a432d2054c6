"""GRMHD-grid plasma on the GPU (fast and slow light, sec. 5) vs the FP64 oracle reading the
same synthetic snapshot arrays.  Needs a GPU."""
import numpy as np
import pytest

from helpers import grid_oracle_scene, grid_plasma_kwargs, rel_err
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu

PIX_TOL = 1e-8
FLUX_TOL = 1e-10
MODEL = scenes.DISK_MODEL
CAM = dict(scenes.SMALL, spin=scenes.TORUS["spin"])


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


@pytest.fixture(scope="module")
def torus():
    return scenes.torus_snapshots(1, n1=64, n2=64, n_modes=128)


@pytest.fixture(scope="module")
def series():
    return scenes.torus_snapshots(12, dt_snap=10.0, n1=48, n2=48, n_modes=128, seed=scenes.SLOW["seed"])


def _ctx(R, cam, fields, meta, slow=0, t0=0.0, **over):
    c = dict(cam)
    c.update(over)
    ctx = R.Context(R.camera_desc(**c))
    ctx.load_plasma(R.plasma_desc(**grid_plasma_kwargs(meta, MODEL, slow, t0)), fields=fields)
    return ctx


def _render(R, ctx, freqs, snap=0):
    import torch

    steps = torch.zeros((ctx.cam.ny, ctx.cam.nx), dtype=torch.int32, device="cuda")
    status = torch.zeros_like(steps)
    img, fl = ctx.render(freqs, steps=steps, status=status, snap=snap)
    torch.cuda.synchronize()
    return img.cpu().numpy(), fl, steps.cpu().numpy(), status.cpu().numpy()


def test_grid_fast_light_fp64_parity(R, ora, torus):
    fields, meta = torus
    cam = dict(CAM, nx=48, ny=40)
    freqs = [86e9, 230e9]
    ctx = _ctx(R, cam, fields, meta)
    img, fl, st, stat = _render(R, ctx, freqs)
    s = grid_oracle_scene(ora, cam, fields, meta, MODEL)
    oimg, ost, ostat = ora.render(s, freqs, t_cam=ctx.cam.t_delay)
    assert np.array_equal(st, ost) and np.array_equal(stat, ostat)
    assert oimg.max() > 0
    for f in range(len(freqs)):
        assert rel_err(img[f], oimg[f]).max() <= PIX_TOL
        assert abs(fl[f] / oimg[f].sum() - 1) <= FLUX_TOL


def test_grid_snapshot_selection_and_device_fields(R, ora, series):
    """render_ex(snap=k) samples snapshot k; fields may come from device memory."""
    import torch

    fields, meta = series
    cam = dict(CAM, nx=20, ny=16)
    ctx = _ctx(R, cam, torch.from_numpy(fields).cuda(), meta)
    img3, _, _, _ = _render(R, ctx, [230e9], snap=3)
    s = grid_oracle_scene(ora, cam, fields, meta, MODEL, snap=3)
    oimg, _, _ = ora.render(s, [230e9], t_cam=ctx.cam.t_delay)
    assert rel_err(img3, oimg).max() <= PIX_TOL
    img0, _, _, _ = _render(R, ctx, [230e9], snap=0)
    assert not np.array_equal(img0, img3)


def test_slow_light_lightcurve_fp64_parity(R, ora, series):
    """One persistent launch over all frames x pixels; every frame matches the oracle's
    slow-light render at that camera time."""
    import torch

    fields, meta = series
    cam = dict(CAM, nx=24, ny=20)
    t0 = -40.0
    ctx = _ctx(R, cam, fields, meta, slow=1, t0=t0)
    t_obs = np.array([0.0, 10.0, 25.0])
    freqs = [230e9]
    imgs = torch.zeros((len(t_obs), 1, cam["ny"], cam["nx"]), dtype=torch.float64, device="cuda")
    fl = ctx.lightcurve(freqs, t_obs, images=imgs)
    imgs = imgs.cpu().numpy()
    s = grid_oracle_scene(ora, cam, fields, meta, MODEL, slow=1, t0=t0)
    prev = None
    for f, t in enumerate(t_obs):
        oimg, _, _ = ora.render(s, freqs, t_cam=t + ctx.cam.t_delay)
        assert rel_err(imgs[f], oimg).max() <= PIX_TOL, f
        assert abs(fl[f, 0] / oimg.sum() - 1) <= FLUX_TOL
        if prev is not None:
            assert fl[f, 0] != prev  # the plasma changes between frames
        prev = fl[f, 0]


def test_fast_light_lightcurve_matches_single_renders(R, series):
    """Fast light: frame f samples snapshot first_frame + f; the batched launch equals the
    per-frame renders bit for bit."""
    fields, meta = series
    cam = dict(CAM, nx=16, ny=16)
    ctx = _ctx(R, cam, fields, meta, slow=0)
    fl = ctx.lightcurve([230e9, 86e9], np.zeros(4), first_frame=5)
    for f in range(4):
        _, fls, _, _ = _render(R, ctx, [230e9, 86e9], snap=5 + f)
        assert np.array_equal(fl[f], fls)
    with pytest.raises(R.RaptorError):
        ctx.lightcurve([230e9], np.zeros(4), first_frame=10)


def test_grid_mixed_precision(R, ora, torus):
    fields, meta = torus
    cam = dict(CAM, nx=48, ny=40)
    ctx = _ctx(R, cam, fields, meta, precision=R.MIXED)
    img, fl, _, _ = _render(R, ctx, [230e9])
    s = grid_oracle_scene(ora, cam, fields, meta, MODEL)
    oimg, _, _ = ora.render(s, [230e9], t_cam=ctx.cam.t_delay)
    assert abs(fl[0] / oimg.sum() - 1) <= 1e-3
    big = oimg[0] > 1e-3 * oimg[0].max()
    assert rel_err(img[0], oimg[0])[big].max() <= 1e-2


def test_grid_headline_sampled_parity(R, ora):
    """The fast-light grid workload at full size (1024^2 pixels, 256 x 256 snapshot), checked
    on seeded sample pixels traced one by one by the oracle."""
    fields, meta = scenes.torus_snapshots(1)
    cam = dict(scenes.HEADLINE)
    ctx = _ctx(R, cam, fields, meta)
    img, fl, st, stat = _render(R, ctx, [230e9])
    s = grid_oracle_scene(ora, cam, fields, meta, MODEL)
    al, be = R.pixel_centres(ctx.cam)
    L = ora.length_unit_cm(cam["mass_msun"])
    D = cam["distance_pc"] * 3.0856775814913673e18
    pix_jy = (al[1] - al[0]) * (be[1] - be[0]) * L**2 / D**2 / 1e-23
    ref = img[0].max()
    for i, j in scenes.sample_pixels(cam["nx"], cam["ny"], 48, seed=3):
        o = ora.trace_ray(s, al[j], be[i], [230e9], t_cam=ctx.cam.t_delay)
        assert st[i, j] == o["steps"] and stat[i, j] == o["status"]
        assert abs(img[0, i, j] - o["I"][0] * pix_jy) <= PIX_TOL * max(o["I"][0] * pix_jy, 1e-12 * ref)
    assert abs(fl[0] - img.sum()) <= 1e-12 * fl[0]
