"""Velocity-Verlet integrator (sec. 2.2.2, RAPTOR_FLAG_VERLET / _VERLET_REEVAL) on the FP64
path against the oracle's Verlet: images, fluxes, step counts and termination codes, and
per-step traces; the flag is refused where it is not built.  Needs a GPU."""
import numpy as np
import pytest

from helpers import oracle_kwargs, rel_err, ring_mask
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu

PIX_TOL = 1e-8
FLUX_TOL = 1e-10


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


def _flags(R, reeval):
    return R.FLAG_VERLET_REEVAL if reeval else R.FLAG_VERLET


@pytest.mark.parametrize("reeval", [False, True])
def test_verlet_image_matches_oracle(R, ora, reeval):
    """48 x 40, a = 0.9, i = 60 deg, two frequencies: the same discrete Verlet scheme on both
    sides (the GPU's closed-form connection against the oracle's generic one)."""
    import torch

    cam = dict(scenes.SMALL, nx=48, ny=40)
    freqs = [1e10, 230e9]
    ctx = R.Context(R.camera_desc(**cam, flags=_flags(R, reeval)))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    steps = torch.zeros((cam["ny"], cam["nx"]), dtype=torch.int32, device="cuda")
    status = torch.zeros_like(steps)
    img, fl = ctx.render(freqs, steps=steps, status=status)
    torch.cuda.synchronize()
    integ = ora.VERLET_REEVAL if reeval else ora.VERLET
    oimg, ost, ostat = ora.render(ora.scene(**oracle_kwargs(cam), integrator=integ), freqs)
    assert np.array_equal(status.cpu().numpy(), ostat)
    assert (steps.cpu().numpy() == ost).mean() > 0.995
    e = rel_err(img.cpu().numpy(), oimg)
    assert e.max() <= PIX_TOL, e.max()
    for f in range(2):
        assert abs(fl[f] / oimg[f].sum() - 1) <= FLUX_TOL
    # against RK4 the image differs by Verlet's truncation error, which shrinks at least 8x
    # when eps shrinks 4x (second order) outside the photon-ring band (inside it the ring's
    # Lyapunov amplification mixes orders)
    al, be = R.pixel_centres(ctx.cam)
    ring = ring_mask(al, be, cam["spin"], cam["incl_deg"], 0.5)

    def rk4_vs_verlet(eps):
        out = []
        for flags in (0, _flags(R, reeval)):
            c = R.Context(R.camera_desc(**dict(cam, eps=eps), flags=flags))
            c.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
            out.append(c.render([230e9])[0][0].cpu().numpy())
        return rel_err(out[1], out[0], floor_frac=1e-6)[~ring].max()

    d1, d4 = rk4_vs_verlet(0.05), rk4_vs_verlet(0.0125)
    assert d1 > 1e-4 and d4 < d1 / 8, (d1, d4)


@pytest.mark.parametrize("reeval", [False, True])
def test_verlet_trace_matches_oracle_per_step(R, ora, reeval):
    cam = dict(scenes.SMALL)
    ctx = R.Context(R.camera_desc(**cam, flags=_flags(R, reeval)))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    s = ora.scene(**oracle_kwargs(cam), integrator=ora.VERLET_REEVAL if reeval else ora.VERLET)
    for al, be in [(5.0, 3.0), (-7.5, 1.0), (2.0, -9.0)]:
        g = ctx.trace_ray(al, be, [230e9], max_rec=5000)
        o = ora.trace_ray(s, al, be, [230e9], max_trace=5000, t_cam=ctx.cam.t_delay)
        assert g["status"] == o["status"] and g["steps"] == o["steps"]
        gt, ot = g["trace"], o["trace"]
        n = min(len(gt), len(ot))
        scale = np.maximum(np.abs(ot[:n, :8]), 1.0)
        assert (np.abs(gt[:n, :8] - ot[:n, :8]) / scale).max() <= 1e-10
        assert abs(g["I"][0] / o["I"][0] - 1) <= PIX_TOL


def test_verlet_refused_outside_fp64(R):
    with pytest.raises(Exception):
        R.Context(R.camera_desc(**scenes.SMALL, precision=R.MIXED, flags=R.FLAG_VERLET))
    ctx = R.Context(R.camera_desc(**scenes.SMALL, flags=R.FLAG_VERLET))
    with pytest.raises(Exception):
        ctx.disk_render(**scenes.THIN_DISK_GEOM)
