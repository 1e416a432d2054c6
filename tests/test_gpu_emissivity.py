"""Emissivity options against the oracle: exact K2 (RAPTOR_FLAG_K2_EXACT; sec. 4.2.2 notes
that evaluating the Bessel function properly changes the flux by a few per cent at most) and
the Theta_e fit-validity mask (plasma theta_e_min), on the FP64 path (<= 1e-8 per pixel,
<= 1e-10 flux) and the mixed path (<= 1e-3 flux).  Needs a GPU."""
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


def _render(R, prec, flags=0, **plasma):
    import torch

    ctx = R.Context(R.camera_desc(**CAM, precision=prec, flags=flags))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA, **plasma))
    img, fl = ctx.render(FREQS)
    torch.cuda.synchronize()
    return img.cpu().numpy(), fl


@pytest.mark.parametrize("k2,mask", [(True, 0.0), (False, 0.5), (False, 2.0), (True, 2.0)])
def test_fp64_options_match_oracle(R, ora, k2, mask):
    img, fl = _render(R, R.FP64, R.FLAG_K2_EXACT if k2 else 0, theta_e_min=mask)
    oimg, _, _ = ora.render(ora.scene(**oracle_kwargs(CAM), k2_exact=int(k2), theta_e_min=mask), FREQS)
    assert rel_err(img, oimg).max() <= 1e-8
    for f in range(len(FREQS)):
        assert abs(fl[f] / oimg[f].sum() - 1) <= 1e-10


def test_option_effects_on_the_flux(R):
    """Exact K2 changes the flux by a few per cent at most at these temperatures.  On this
    scene (Theta_e = 10/r) the fit's own limit Theta_e = 0.5 (r > 20 M) masks nothing that
    emits at these frequencies; a mask at Theta_e = 2 (r > 5 M) removes emission: the flux
    never grows, and at 10 GHz, where the emission reaches out furthest, it drops."""
    img0, fl0 = _render(R, R.FP64)
    _, flk = _render(R, R.FP64, R.FLAG_K2_EXACT)
    _, flh = _render(R, R.FP64, theta_e_min=0.5)
    _, flm = _render(R, R.FP64, theta_e_min=2.0)
    assert np.all(np.abs(flk / fl0 - 1) < 0.1) and np.any(np.abs(flk / fl0 - 1) > 1e-4)
    assert np.all(np.abs(flh / fl0 - 1) < 1e-6)
    assert np.all(flm <= fl0 * (1 + 1e-12)) and flm[0] < fl0[0] * (1 - 1e-2)


@pytest.mark.parametrize("flags", [0, "df64"])
def test_mixed_path_with_mask_and_k2(R, flags):
    """The mixed path honours both options within its 1e-3 flux bound of the FP64 path."""
    fl = R.FLAG_INNER_DF64 if flags else 0
    for k2, mask in [(False, 2.0), (True, 0.0)]:
        f = fl | (R.FLAG_K2_EXACT if k2 else 0)
        _, fm = _render(R, R.MIXED, f, theta_e_min=mask)
        _, fr = _render(R, R.FP64, R.FLAG_K2_EXACT if k2 else 0, theta_e_min=mask)
        for i in range(len(FREQS)):
            if fr[i] > 1e-30:
                assert abs(fm[i] / fr[i] - 1) <= 1e-3, (k2, mask, i)
