"""Optical-depth early exit (camera tau_cut; the paper's tau_cutoff = ln 1000, Table 2): the
FP64 path against the oracle with the cut (termination codes including 'thick', images,
fluxes), the cut's effect (fewer steps, flux change below exp(-tau_cut) of the total), and
the mixed path within its flux bound.  Needs a GPU."""
import math

import numpy as np
import pytest

from helpers import oracle_kwargs, rel_err
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu

TAU_CUT = math.log(1000.0)
CAM = dict(scenes.SMALL, nx=48, ny=40, tau_cut=TAU_CUT)
FREQS = [1e10]  # the cut applies to the smallest optical depth over the frequencies


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


def _render(R, cam, prec=None, flags=0):
    import torch

    ctx = R.Context(R.camera_desc(**cam, **({} if prec is None else {"precision": prec}), flags=flags))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    steps = torch.zeros((cam["ny"], cam["nx"]), dtype=torch.int32, device="cuda")
    status = torch.zeros_like(steps)
    img, fl = ctx.render(FREQS, steps=steps, status=status)
    torch.cuda.synchronize()
    return img.cpu().numpy(), fl, steps.cpu().numpy(), status.cpu().numpy()


def test_tau_cut_fp64_matches_oracle(R, ora):
    img, fl, st, stat = _render(R, CAM)
    oimg, ost, ostat = ora.render(ora.scene(**oracle_kwargs(CAM)), FREQS)
    assert (stat == ora.THICK).sum() >= 3
    assert np.array_equal(stat, ostat) and np.array_equal(st, ost)
    assert rel_err(img, oimg).max() <= 1e-8
    for f in range(len(FREQS)):
        assert abs(fl[f] / oimg[f].sum() - 1) <= 1e-10


def test_tau_cut_effect_and_mixed_path(R):
    img, fl, st, stat = _render(R, CAM)
    cam_inf = dict(CAM, tau_cut=float("inf"))
    img0, fl0, st0, stat0 = _render(R, cam_inf)
    thick = stat == 2
    assert (st[thick] < st0[thick]).all() and (st[~thick] == st0[~thick]).all()
    # what the cut leaves out is attenuated by at least exp(-tau_cut) = 1e-3
    assert np.all(fl <= fl0 * (1 + 1e-12)) and np.all(fl >= fl0 * (1 - 1e-3))
    for flags in (0, R.FLAG_INNER_DF64):
        _, fm, _, sm = _render(R, CAM, R.MIXED, flags)
        assert (sm == 2).sum() >= 1
        assert np.all(np.abs(fm / fl - 1) <= 1e-3)
