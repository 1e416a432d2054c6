"""Forward formal-solution transfer (RAPTOR_FLAG_FORWARD_RT, sec. 3, Eq. 34 from each ray's
far end) on the FP64 path: against the oracle's forward scheme (<= 1e-8 per pixel, <= 1e-10
flux, equal terminations, also with the optical-depth cut-off and per traced ray), against
the library's own backward scheme to rounding, and its limits.  Needs a GPU."""
import math

import numpy as np
import pytest

from helpers import oracle_kwargs, rel_err
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu

CAM = dict(scenes.SMALL, nx=40, ny=32)
FREQS = [1e10, 230e9, 1e12]


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


def _render(R, cam, flags):
    import torch

    ctx = R.Context(R.camera_desc(**cam, flags=flags))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    st = torch.zeros((cam["ny"], cam["nx"]), dtype=torch.int32, device="cuda")
    stat = torch.zeros_like(st)
    img, fl = ctx.render(FREQS, steps=st, status=stat)
    torch.cuda.synchronize()
    return ctx, img.cpu().numpy(), fl, st.cpu().numpy(), stat.cpu().numpy()


@pytest.mark.parametrize("tau_cut", [float("inf"), math.log(1000.0)])
def test_forward_matches_oracle_and_backward(R, ora, tau_cut):
    cam = dict(CAM, tau_cut=tau_cut)
    _, img, fl, st, stat = _render(R, cam, R.FLAG_FORWARD_RT)
    oimg, ost, ostat = ora.render(ora.scene(**oracle_kwargs(cam), rt_scheme=1), FREQS)
    assert np.array_equal(stat, ostat) and np.array_equal(st, ost)
    assert rel_err(img, oimg).max() <= 1e-8
    for f in range(len(FREQS)):
        assert abs(fl[f] / oimg[f].sum() - 1) <= 1e-10
    _, bimg, bfl, bst, bstat = _render(R, cam, 0)
    assert np.array_equal(bstat, stat) and np.array_equal(bst, st)
    assert rel_err(img, bimg).max() <= 1e-12
    assert np.all(np.abs(fl / bfl - 1) <= 1e-12)


def test_forward_trace_matches_oracle(R, ora):
    ctx = R.Context(R.camera_desc(**CAM, flags=R.FLAG_FORWARD_RT))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    s = ora.scene(**oracle_kwargs(CAM), rt_scheme=1)
    for al, be in [(5.0, 3.0), (-3.0, 0.5), (0.31, -7.9)]:
        g = ctx.trace_ray(al, be, FREQS, max_rec=10)
        o = ora.trace_ray(s, al, be, FREQS, t_cam=ctx.cam.t_delay)
        assert g["status"] == o["status"] and g["steps"] == o["steps"]
        assert np.all(np.abs(g["I"] - o["I"]) <= 1e-8 * np.abs(o["I"]) + 1e-300)


def test_forward_limits(R):
    with pytest.raises(Exception):
        R.Context(R.camera_desc(**CAM, precision=R.MIXED, flags=R.FLAG_FORWARD_RT))
    ctx = R.Context(R.camera_desc(**CAM, flags=R.FLAG_FORWARD_RT))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    with pytest.raises(Exception):
        ctx.render(list(np.logspace(10, 12, 5)))
