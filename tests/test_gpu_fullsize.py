"""The grid workloads at the sizes and in the launch configuration the benchmark times: the
fast-light torus image (1024^2 pixels, 256 x 256 snapshot) and the slow-light light curve
(100 frames of 256^2 over 100 snapshots 10 M apart, one batched launch sequence), through the
FP64, mixed (double-float inner steps) and learned paths.  Fluxes of the mixed and learned
paths against the FP64 GPU path (<= 1e-3), every pixel of the grid image outside 0.5 M of the
critical curve against the FP64 GPU image (<= 1e-2), seeded sample pixels (and frames)
traced one by one by the oracle (FP64 <= 1e-8; mixed and learned <= 1e-2 outside 0.5 M of
the critical curve).  Needs a GPU."""
import numpy as np
import pytest

from helpers import grid_oracle_scene, grid_plasma_kwargs, near_ring
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu

MODEL = scenes.DISK_MODEL
FLUX_TOL = 1e-3
PIX_TOL = 1e-2


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


@pytest.fixture(scope="module")
def trained(R):
    import torch

    ctx = R.Context(R.camera_desc(**scenes.SMALL, precision=R.MIXED_MLP))
    ctx.surrogate_handoff(30)  # the torus's fine structure wants the earlier hand-off
    x, y = ctx.surrogate_generate(1_000_000, seed=0x1801104520000005)
    ctx.surrogate_init(y, seed=7)
    ctx.surrogate_train(x, y, 16000, lr=2e-3, lr_final=2e-5, seed=11)
    torch.cuda.synchronize()
    return ctx.surrogate_get()


PATHS = [("fp64", "FP64", 0), ("mixed_df", "MIXED", "df"), ("mlp_df", "MIXED_MLP", "df")]


def _ctx(R, cam, fields, meta, name, trained, slow=0, t0=0.0):
    _, prec, fl = next(p for p in PATHS if p[0] == name)
    ctx = R.Context(R.camera_desc(**cam, precision=getattr(R, prec), flags=R.FLAG_INNER_DF64 if fl else 0))
    ctx.load_plasma(R.plasma_desc(**grid_plasma_kwargs(meta, MODEL, slow, t0)), fields=fields)
    if name == "mlp_df":
        ctx.surrogate_set(trained)
    return ctx


def _band(al, be, cam, width=0.5):
    """Pixels within `width` M of the critical curve (nearest vertex of a densely sampled
    Bardeen curve by a k-d tree)."""
    from scipy.spatial import cKDTree

    from helpers import bardeen_critical_curve

    A, B = np.meshgrid(al, be)
    d, _ = cKDTree(bardeen_critical_curve(cam["spin"], cam["incl_deg"], 20000)).query(np.stack([A.ravel(), B.ravel()], 1))
    return (d < width).reshape(A.shape)


def _pix_jy(R, ora, ctx, cam):
    al, be = R.pixel_centres(ctx.cam)
    L = ora.length_unit_cm(cam["mass_msun"])
    D = cam["distance_pc"] * 3.0856775814913673e18
    return al, be, (al[1] - al[0]) * (be[1] - be[0]) * L**2 / D**2 / 1e-23


def test_grid_image_full_size_all_paths(R, ora, trained):
    import torch

    fields, meta = scenes.torus_snapshots(1)
    cam = dict(scenes.HEADLINE)
    freqs = [230e9]
    s = grid_oracle_scene(ora, cam, fields, meta, MODEL)
    pix = scenes.sample_pixels(cam["nx"], cam["ny"], 40, seed=1024)
    fl64 = img64 = band = None
    for name, _, _ in PATHS:
        ctx = _ctx(R, cam, fields, meta, name, trained)
        img, fl = ctx.render(freqs)
        torch.cuda.synchronize()
        img = img.cpu().numpy()[0]
        al, be, pj = _pix_jy(R, ora, ctx, cam)
        if name == "fp64":
            fl64, img64 = fl, img
            band = _band(al, be, cam)
        else:
            assert abs(fl[0] / fl64[0] - 1) <= FLUX_TOL, (name, fl[0] / fl64[0] - 1)
            # every pixel outside the band against the FP64 GPU image (itself within 1e-8 of
            # the oracle): relative for pixels above 1e-6 of the peak, absolute below
            pk = img64.max()
            bright = np.abs(img64) >= 1e-6 * pk
            d = np.abs(img - img64)
            rel = d / np.maximum(np.abs(img64), 1e-300)
            m = ~band & bright
            over = rel[m] > PIX_TOL
            print(f"grid 1024^2 {name} vs FP64 outside the band: max rel {rel[m].max():.2e}, "
                  f"{int(over.sum())} of {int(m.sum())} pixels above {PIX_TOL:g}, brightest of them "
                  f"{(img64[m][over].max() / pk if over.any() else 0):.1e} of the peak; fainter pixels "
                  f"within {d[~band & ~bright].max() / pk:.1e} of the peak")
            if name == "mixed_df":
                assert rel[m].max() <= PIX_TOL, name
                assert d[~band & ~bright].max() <= 1e-8 * pk, name
            else:
                # the network's angular error at the hand-off carries over to the path at the
                # torus, whose sharp inner edge changes some pixels by 3-10 % per 1e-3 M of
                # image-plane offset: the per-pixel bound holds for all but ~0.01 % of the
                # pixels with the 30-step hand-off (0.1 % with 60; measured), which this
                # checks with margin; pixels fainter than 1e-6 of the peak within 1e-6 of it
                assert over.mean() <= 1e-3, (name, over.mean())
                assert d[~band & ~bright].max() <= 1e-6 * pk, name
        keep = ~near_ring(al[pix[:, 1]], be[pix[:, 0]], cam["spin"], cam["incl_deg"], 0.5)
        tol = 1e-8 if name == "fp64" else PIX_TOL
        peak = img.max()
        for i, j in (pix if name == "fp64" else pix[keep]):
            ov = ora.trace_ray(s, al[j], be[i], freqs, t_cam=ctx.cam.t_delay)["I"][0] * pj
            floor = 1e-12 if name == "fp64" else 1e-6
            assert abs(img[i, j] - ov) <= tol * max(abs(ov), floor * peak), (name, i, j)


def test_lightcurve_full_size_all_paths(R, ora, trained):
    """100 frames of 256^2 at 230 GHz, slow light over 100 snapshots (t0 = -50 M, frames
    10 M apart) in one batched launch sequence, as the benchmark runs it."""
    import torch

    n = 100
    fields, meta = scenes.torus_snapshots(n, dt_snap=10.0, seed=scenes.SLOW["seed"])
    cam = dict(scenes.HEADLINE, nx=256, ny=256)
    freqs = [230e9]
    t_obs = 10.0 * np.arange(n)
    s = grid_oracle_scene(ora, cam, fields, meta, MODEL, slow=1, t0=-50.0)
    rng = np.random.default_rng(256)
    samples = [(int(f), int(i), int(j)) for f, i, j in zip(rng.integers(0, n, 16), rng.integers(0, 256, 16),
                                                           rng.integers(0, 256, 16))]
    fl64 = None
    for name, _, _ in PATHS:
        ctx = _ctx(R, cam, fields, meta, name, trained, slow=1, t0=-50.0)
        imgs = torch.zeros((n, 1, cam["ny"], cam["nx"]), dtype=torch.float64, device="cuda")
        fl = ctx.lightcurve(freqs, t_obs, images=imgs)
        imgs = imgs.cpu().numpy()
        if name == "fp64":
            fl64 = fl
        else:
            rel = np.abs(fl[:, 0] / fl64[:, 0] - 1)
            assert rel.max() <= FLUX_TOL, (name, rel.max())
        al, be, pj = _pix_jy(R, ora, ctx, cam)
        tol = 1e-8 if name == "fp64" else PIX_TOL
        for f, i, j in samples:
            if name != "fp64" and near_ring(al[[j]], be[[i]], cam["spin"], cam["incl_deg"], 0.5)[0]:
                continue
            ov = ora.trace_ray(s, al[j], be[i], freqs, t_cam=t_obs[f] + ctx.cam.t_delay)["I"][0] * pj
            peak = imgs[f, 0].max()
            floor = 1e-12 if name == "fp64" else 1e-6
            assert abs(imgs[f, 0, i, j] - ov) <= tol * max(abs(ov), floor * peak), (name, f, i, j)


def test_large_image_mixed_and_learned(R, ora, trained):
    """4096^2 (16.8 M rays, ~35 GB of hand-off queues): no index overflows in the queues,
    the network's buffers or the reductions.  Fluxes of the mixed and learned paths against
    the FP64 GPU path, seeded pixels outside the photon-ring band against the oracle."""
    import torch

    cam = dict(scenes.HEADLINE, nx=4096, ny=4096)
    freqs = [230e9]
    ref = R.Context(R.camera_desc(**cam))
    ref.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    _, fl64 = ref.render(freqs, image=torch.empty((1, 4096, 4096), dtype=torch.float64, device="cuda"))
    ref.close()
    s = ora.scene(**__import__("helpers").oracle_kwargs(cam))
    pix = scenes.sample_pixels(4096, 4096, 32, seed=4096)
    for prec in ("MIXED", "MIXED_MLP"):
        ctx = R.Context(R.camera_desc(**cam, precision=getattr(R, prec), flags=R.FLAG_INNER_DF64))
        ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
        if prec == "MIXED_MLP":
            ctx.surrogate_set(trained)
        img, fl = ctx.render(freqs)
        torch.cuda.synchronize()
        assert abs(fl[0] / fl64[0] - 1) <= FLUX_TOL, (prec, fl[0] / fl64[0] - 1)
        st = ctx.stats()
        assert st["rays"] == 4096 * 4096 and st["errors"] == 0
        al, be, pj = _pix_jy(R, ora, ctx, cam)
        keep = ~near_ring(al[pix[:, 1]], be[pix[:, 0]], cam["spin"], cam["incl_deg"], 0.5)
        peak = float(img.max())
        for i, j in pix[keep]:
            ov = ora.trace_ray(s, al[j], be[i], freqs, t_cam=ctx.cam.t_delay)["I"][0] * pj
            g = float(img[0, i, j])
            assert abs(g - ov) <= PIX_TOL * max(abs(ov), 1e-6 * peak), (prec, i, j)
        del img
        ctx.close()
        torch.cuda.empty_cache()
