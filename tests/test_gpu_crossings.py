"""Learned equatorial crossings (the surrogate's thin-disk outputs) and the learned thin disk:
integrator-generated crossings against the FP64 oracle, the library's backward pass against
the FP64 network oracle, held-out accuracy of the trained network, and the learned disk image
against the exact FP64 disk (sec. 4.2.1) and the oracle.  Needs a GPU."""
import time

import numpy as np
import pytest

from helpers import near_ring, oracle_kwargs
from oracle import mlp
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu

DISK = dict(scenes.THIN_DISK_GEOM)
RATIO_TOL = 1e-2    # per pixel, outside the fallback band (the learned paths' per-pixel bound)
SPEC_TOL = 1e-2     # line spectrum: total and L1 distance of the normalised spectra


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


@pytest.fixture(scope="module")
def trained(R):
    """A crossing network trained on the learned workload's range (a in [0, 0.99], i in
    [5, 85] deg, +-20 M), shared by the tests below."""
    import torch

    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    x, y = ctx.crossings_generate(2_000_000, seed=21)
    ctx.crossings_init(y, seed=7)
    ctx.crossings_train(x, y, 16000, lr=2e-3, lr_final=2e-5, seed=11)
    torch.cuda.synchronize()
    return ctx.crossings_get()


def test_crossing_data_is_the_integrator(R, ora):
    """The generator's crossings (radius, affine length) equal the oracle's FP64 trace, and
    each ratio equals the oracle's thin-disk E_obs/E_em for a disk ring around that radius;
    the targets are the raw values as documented (ln r, increments of lambda from the
    straight ray's length, NaN ratio inside the ISCO)."""
    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    x, y, z = ctx.crossings_generate(96, seed=3, raw=True)
    xs, ys, zs = x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy()
    n_cross = 0
    for i in range(96):
        al, be, a, inc = map(float, xs[i])
        s = ora.scene(a=a, incl_deg=inc)
        o = ora.disk_crossings(s, al, be, max_n=4)
        nc = len(o["r"])
        assert int(zs[i, 0::4].sum()) == nc, (i, zs[i], o)
        for n in range(4):
            if n >= nc:
                assert ys[i, 4 * n] == 0 and np.all(np.isnan(ys[i, 4 * n + 1:4 * n + 4]))
                continue
            n_cross += 1
            r, lam = zs[i, 4 * n + 1], zs[i, 4 * n + 2]
            assert abs(r / o["r"][n] - 1) <= 1e-9, (i, n, r, o["r"][n])
            assert abs(lam / o["lam"][n] - 1) <= 1e-9, (i, n, lam, o["lam"][n])
            assert ys[i, 4 * n] == 1
            if n:
                assert abs(ys[i, 4 * n + 1] - np.log(r)) <= 1e-15 * abs(np.log(r)) + 1e-15
            prev = zs[i, 4 * n - 2] if n else None
            if prev is not None:
                assert abs(ys[i, 4 * n + 2] - (lam - prev)) <= 1e-9 * lam
            d = ora.disk_ray(s, al, be, r_in=r * (1 - 1e-7), r_out=r * (1 + 1e-7), max_cross=10)
            if np.isnan(zs[i, 4 * n + 3]):
                # no timelike circular orbit there (inside the photon orbit): the oracle's disk
                # ray ends in its error status at that crossing
                assert d["status"] == ora.ERROR, (i, n, d)
                continue
            assert d["status"] == ora.DISK_HIT and d["order"] == n + 1, (i, n, d)
            assert abs(zs[i, 4 * n + 3] / d["ratio"] - 1) <= 1e-9
            r_isco = ora.r_isco(a)
            if r >= r_isco:
                assert ys[i, 4 * n + 3] == zs[i, 4 * n + 3]
            else:
                assert np.isnan(ys[i, 4 * n + 3])
        # the first crossing against the straight ray's (camera height / descent rate; radius
        # at the plane, softened by 3 M), which the generator computes in FP32
        if nc:
            x0, k0 = ora.camera(s, al, be)
            inc_r = np.radians(inc)
            rc, sn, cs = x0[1], np.sin(inc_r), np.cos(inc_r)
            vx, vy, vz = k0[1] * sn + rc * k0[2] * cs, rc * sn * k0[3], k0[1] * cs - rc * k0[2] * sn
            lam_flat = -rc * cs / vz
            X, Y = rc * sn + vx * lam_flat, vy * lam_flat
            assert abs((zs[i, 2] - ys[i, 2]) / lam_flat - 1) <= 1e-5
            assert abs((np.log(zs[i, 1]) - ys[i, 1]) - 0.5 * np.log(X * X + Y * Y + 9)) <= 1e-3
    assert n_cross >= 96


def test_crossing_backward_matches_fp64_oracle(R):
    """Gradient of the crossing loss from the library's kernels (BF16 hidden layers) against
    the FP64 chain rule of the network oracle, per tensor, at the initial weights: 1e-2
    relative L2 (BF16's 8-bit mantissa), loss within 2e-3."""
    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    x, y = ctx.crossings_generate(4096, seed=13)
    ctx.crossings_init(y, seed=17)
    P = ctx.crossings_get().astype(np.float64)
    xb, yb = x[:512].contiguous(), y[:512].contiguous()
    g, L = ctx.crossings_grad(xb, yb)
    xo, yo = xb.cpu().numpy().astype(np.float64), yb.cpu().numpy()
    go = mlp.x_grad(P, xo, yo)
    Lo = mlp.x_loss(P, xo, yo)
    assert abs(L / Lo - 1) < 2e-3, (L, Lo)
    for a, b in [(mlp.W1, mlp.B1), (mlp.B1, mlp.W2), (mlp.W2, mlp.B2), (mlp.B2, mlp.W3), (mlp.W3, mlp.B3),
                 (mlp.B3, mlp.XW4), (mlp.XW4, mlp.XB4), (mlp.XB4, mlp.XNORM)]:
        e = np.linalg.norm(g[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
        assert e < 1e-2, (a, b, e)


def test_crossings_generalise_to_held_out_rays(R, ora, trained):
    """Held-out rays of one scene (a = 0.9375, i = 60 deg, +-20 M; not in the training set):
    outside the 0.5 M band around the critical curve the predicted crossing count is right
    for nearly every ray; the first crossing's radius, length and E_obs/E_em are within the
    learned paths' 1e-2 per-result bound at the median (99 % of the rays within 2e-2; the image
    test below holds every disk pixel to 1e-2), the later crossings (rays that pass close to
    the hole) within a few per cent."""
    import torch

    cam = dict(scenes.SMALL, spin=0.9375)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.crossings_set(trained)
    x, y, z = ctx.crossings_generate(50_000, seed=0xABCDEF, spin=(0.9375, 0.9375), incl=(60.0, 60.0), raw=True)
    pred = ctx.crossings_eval(x)
    torch.cuda.synchronize()
    xs, zs, ps = x.cpu().numpy().astype(np.float64), z.cpu().numpy(), pred.cpu().numpy()
    keep = ~near_ring(xs[:, 0], xs[:, 1], 0.9375, 60.0, 0.5)
    zs, ps = zs[keep], ps[keep]
    pres_true = zs[:, 0::4] > 0.5
    pres_pred = ps[:, 0::4] > 0.5
    assert np.mean(np.all(pres_true == pres_pred, axis=1)) >= 0.995
    both = pres_true & pres_pred
    r_isco = ora.r_isco(0.9375)

    def errs(c, sel):
        m = both[:, c] & sel
        er = np.abs(ps[m, 4 * c + 1] / zs[m, 4 * c + 1] - 1)
        el = np.abs(ps[m, 4 * c + 2] / zs[m, 4 * c + 2] - 1)
        mg = m & (zs[:, 4 * c + 1] >= r_isco)
        eg = np.abs(ps[mg, 4 * c + 3] / zs[mg, 4 * c + 3] - 1)
        return er, el, eg

    er, el, eg = errs(0, np.ones(len(zs), bool))
    print("first crossing: r median %.2e p99 %.2e, lambda p99 %.2e, ratio median %.2e p99 %.2e"
          % (np.median(er), np.quantile(er, 0.99), np.quantile(el, 0.99), np.median(eg), np.quantile(eg, 0.99)))
    assert np.median(er) < 3e-3 and np.median(eg) < 3e-3
    assert np.quantile(er, 0.99) < 2e-2 and np.quantile(eg, 0.99) < 2e-2 and np.quantile(el, 0.99) < 1e-3
    later = [np.concatenate(v) for v in zip(*[errs(c, np.ones(len(zs), bool)) for c in (1, 2, 3)])]
    print("later crossings: r median %.2e, ratio median %.2e (%d)" % (np.median(later[0]), np.median(later[2]),
                                                                      len(later[0])))
    assert np.median(later[0]) < 5e-2 and np.median(later[2]) < 5e-2


def _disk(R, ctx, learned, **kw):
    import torch

    out = ctx.disk_render(**DISK, learned=learned, **kw)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


@pytest.mark.parametrize("spin,incl", [(0.9375, 30.0), (0.5, 60.0)])
def test_learned_disk_matches_fp64_disk_and_oracle(R, ora, trained, spin, incl):
    """Learned thin disk (256^2, +-16 M) against the exact FP64 disk: with the FP64 fallback
    the fallback pixels equal it bit for bit (the same kernel), with the double-float fallback
    (the default) they agree on hit and order for >= 99.9 % and on E_obs/E_em within
    rounding amplified near the photon orbit; the learned pixels agree on hit and order for
    >= 99.5 % of the
    pixels (the rest lie at the disk's edges, where a radius error moves the crossing across
    r_in or r_out) and on E_obs/E_em within 1e-2; the line spectrum within 1e-2; sampled
    pixels against the oracle one by one."""
    cam = dict(scenes.THIN_DISK, spin=spin, incl_deg=incl, nx=256, ny=256)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.crossings_set(trained)
    f = _disk(R, ctx, False)
    ctx.crossings_config(1.0, fallback_df64=False)
    g64 = _disk(R, ctx, True)
    ctx.crossings_config(1.0, fallback_df64=True)
    g = _disk(R, ctx, True)
    fb = g["steps"] > 0
    assert fb.any() and (~fb).sum() > 0.8 * fb.size
    assert np.array_equal(g64["steps"] > 0, fb)
    # FP64 fallback: the FP64 disk's own values; double-float fallback: the same hits, ratios
    # within rounding amplified by the near-critical orbits
    for k in ("ratio", "intensity", "order", "status", "steps"):
        assert np.array_equal(g64[k][fb], f[k][fb]), k
        assert np.array_equal(g64[k][~fb], g[k][~fb]), k
    same = fb & (g["order"] == f["order"])
    assert same.sum() >= 0.999 * fb.sum(), (same.sum(), fb.sum())
    both = same & (f["order"] > 0)
    d = np.abs(g["ratio"][both] / f["ratio"][both] - 1)
    print("double-float fallback: %d pixels, order agreement %.5f, ratio diff median %.1e max %.1e"
          % (fb.sum(), same.sum() / fb.sum(), np.median(d), d.max()))
    assert np.median(d) <= 1e-9 and d.max() <= RATIO_TOL
    nb = ~fb
    agree = (g["order"][nb] == f["order"][nb])
    assert agree.mean() >= 0.995, agree.mean()
    hit = nb & (f["order"] > 0) & (g["order"] == f["order"])
    assert hit.sum() > 1000
    rel = np.abs(g["ratio"][hit] / f["ratio"][hit] - 1)
    print("learned disk a=%g i=%g: fallback %.3f, order agreement %.4f, ratio err max %.2e p99 %.2e"
          % (spin, incl, fb.mean(), agree.mean(), rel.max(), np.quantile(rel, 0.99)))
    assert rel.max() <= RATIO_TOL, rel.max()
    sf, sg = f["spectrum"], g["spectrum"]
    assert abs(sg.sum() / sf.sum() - 1) <= SPEC_TOL, (sg.sum(), sf.sum())
    # shape: a ratio error of ~1e-3 moves a pixel across an edge of the 0.022-wide bins, so
    # the shape is compared on groups of four bins, and by the line's centroid
    c = 0.5 * (g["edges"][1:] + g["edges"][:-1])
    assert abs((sg * c).sum() / sg.sum() / ((sf * c).sum() / sf.sum()) - 1) <= 1e-3
    s4g, s4f = sg.reshape(-1, 4).sum(1), sf.reshape(-1, 4).sum(1)
    l1 = np.abs(s4g / s4g.sum() - s4f / s4f.sum()).sum()
    print("spectrum: total %.2e, grouped L1 %.3f" % (sg.sum() / sf.sum() - 1, l1))
    assert l1 <= 2 * SPEC_TOL, l1
    # oracle, pixel by pixel, on a seeded sample of the learned pixels that hit
    s = ora.scene(**oracle_kwargs(cam))
    al, be = R.pixel_centres(R.camera_desc(**cam))
    rows, cols = np.nonzero(hit)
    pick = np.random.default_rng(77).choice(len(rows), 24, replace=False)
    for q in pick:
        i, j = rows[q], cols[q]
        d = ora.disk_ray(s, al[j], be[i], **DISK)
        assert d["status"] == ora.DISK_HIT and d["order"] == g["order"][i, j]
        assert abs(g["ratio"][i, j] / d["ratio"] - 1) <= RATIO_TOL


def test_learned_disk_gain(R, trained):
    """What the crossing network buys on the thin-disk workload's 1024^2 image: the learned
    disk (network for ~all pixels, exact integration near the critical curve) against the FP64
    disk, same camera."""
    import torch

    cam = dict(scenes.THIN_DISK, spin=0.9375)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.crossings_set(trained)

    def run(learned):
        _disk(R, ctx, learned)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _disk(R, ctx, learned)
        torch.cuda.synchronize()
        return time.perf_counter() - t

    t_f, t_l = run(False), run(True)
    assert t_l < 0.5 * t_f, (t_l, t_f)


def test_learned_disk_argument_checks(R, trained):
    cam = dict(scenes.THIN_DISK, spin=0.0, nx=32, ny=32)
    ctx = R.Context(R.camera_desc(**cam))
    with pytest.raises(R.RaptorError) as e:
        ctx.disk_render(**DISK, learned=True)
    assert e.value.status == R.EUNSUPPORTED
    ctx.crossings_set(trained)
    with pytest.raises(R.RaptorError) as e:
        ctx.disk_render(r_in=4.0, r_out=15.0, learned=True)
    assert e.value.status == R.EUNSUPPORTED
    for bad in (-0.1, float("nan"), float("inf")):
        with pytest.raises(R.RaptorError) as e:
            ctx.crossings_config(bad)
        assert e.value.status == R.EINVAL
    from paper_1801_10452_b300 import lib
    assert lib().raptor_crossings_config(ctx.handle, 1.0, 2) == R.EINVAL
    for bad in ((-0.1, 0.01), (1.0, float("nan"))):
        with pytest.raises(R.RaptorError) as e:
            ctx.crossings_confidence(*bad)
        assert e.value.status == R.EINVAL
    ctx.disk_render(**DISK, learned=True)
    # a camera outside the network's training range (spin in [0, 0.99], inclination in
    # [5, 85] deg) is refused rather than extrapolated
    for over in (dict(spin=-0.5), dict(incl_deg=89.0)):
        out = R.Context(R.camera_desc(**dict(cam, **over)))
        out.crossings_set(trained)
        with pytest.raises(R.RaptorError) as e:
            out.disk_render(r_in=8.0, r_out=15.0, learned=True)
        assert e.value.status == R.EUNSUPPORTED


def test_learned_disk_band_zero_and_wide(R, trained):
    """The fallback band sets which pixels are integrated exactly: band 0 leaves only the
    shadow (inside the critical curve) to the integrator, a wide band more pixels, and every
    fallback pixel equals the FP64 disk."""
    cam = dict(scenes.THIN_DISK, spin=0.5, nx=128, ny=128)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.crossings_set(trained)
    f = _disk(R, ctx, False)
    frac = []
    for band in (0.0, 1.0, 3.0):
        ctx.crossings_config(band, fallback_df64=False)
        g = _disk(R, ctx, True)
        fb = g["steps"] > 0
        frac.append(fb.mean())
        assert np.array_equal(g["ratio"][fb], f["ratio"][fb]) and np.array_equal(g["order"][fb], f["order"][fb])
    assert 0 < frac[0] < frac[1] < frac[2] < 1, frac


def _bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("n", [1, 3001, 70000])
def test_crossing_network_inference_kernels(R, trained, n):
    """Inference of the 16-output network on tcgen05 (default; its output layer reduced in
    two rounds of 8) and on mma.sync against the FP64 network oracle with the same BF16
    roundings, on 1 row, a ragged 23.4 tiles and 547 tiles: decoded radii (ln r, the first
    crossing's against the straight ray's) and presence probabilities agree to FP32
    accumulation, apart from rare BF16 rounding flips of an activation."""
    import torch

    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    ctx.crossings_set(trained)
    P = trained.astype(np.float64)
    x, _ = ctx.crossings_generate(n, seed=43)
    p = mlp.x_unpack(P)
    xn = (x.cpu().numpy().astype(np.float64) - p["shift"]) * p["scale"]
    h1 = _bf16(mlp.silu(xn @ p["W1"].T + p["b1"]))
    h2 = _bf16(mlp.silu(h1 @ _bf16(p["W2"]).T + p["b2"]))
    h3 = _bf16(mlp.silu(h2 @ _bf16(p["W3"]).T + p["b3"]))
    ref = h3 @ p["W4"].T + p["b4"]
    prob_ref = 1 / (1 + np.exp(-ref[:, 0::4]))
    outs = {}
    for kind in (R.MLP_TCGEN05, R.MLP_MMA_SYNC):
        ctx.surrogate_kernel(kind)
        pr = ctx.crossings_eval(x)
        torch.cuda.synchronize()
        pr = pr.cpu().numpy()
        outs[kind] = pr
        # ln r of crossings 2-4 is the normalised output itself: compare in output units
        lnr = (np.log(pr[:, 5::4]) - p["mu"][5::4]) / p["sd"][5::4]
        d = np.abs(lnr - ref[:, 5::4])
        # FP32 accumulation plus the rare BF16 flips, which the mean and the tail carry; the
        # later crossings' radii spread less than the state network's outputs, so a flip moves
        # them further in normalised units.  The 70,000-row case measured on tcgen05: mean
        # 3.1e-5, 99.9th percentile 6.4e-3, largest 0.24 (a row with several flips).
        assert d.mean() < 5e-5 and np.quantile(d, 0.999) < 1e-2 and d.max() < 0.3, (kind, d.max(), d.mean())
        dp = np.abs(pr[:, 0::4] - prob_ref)
        assert dp.mean() < 1e-5 and dp.max() < 0.05, (kind, dp.max())
    assert np.abs(outs[R.MLP_TCGEN05][:, 1::4] / outs[R.MLP_MMA_SYNC][:, 1::4] - 1).mean() < 1e-4


def test_learned_disk_retrograde(R, ora):
    """Retrograde spins (the disk workload's a < 0): a crossing network trained on
    a in [-0.99, 0] (inputs normalised over that range) draws the a = -0.5 disk (i = 30 deg,
    256^2) like the FP64 disk: hit order agrees on >= 99.5 % of the learned pixels, every
    compared E_obs/E_em within 1e-2, line flux within 1e-2; sampled pixels against the
    oracle."""
    import torch

    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    x, y = ctx.crossings_generate(2_000_000, seed=23, spin=(-0.99, 0.0))
    ctx.crossings_init(y, seed=7, inputs=x)
    ctx.crossings_train(x, y, 16000, lr=2e-3, lr_final=2e-5, seed=11)
    torch.cuda.synchronize()
    P = ctx.crossings_get()
    cam = dict(scenes.THIN_DISK, spin=-0.5, nx=256, ny=256)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.crossings_set(P)
    f = _disk(R, ctx, False)
    g = _disk(R, ctx, True)
    nb = g["steps"] == 0
    agree = g["order"][nb] == f["order"][nb]
    hit = nb & (f["order"] > 0) & (g["order"] == f["order"])
    rel = np.abs(g["ratio"][hit] / f["ratio"][hit] - 1)
    print("retrograde learned disk: order agreement %.4f, ratio err max %.2e p99 %.2e (%d pixels)"
          % (agree.mean(), rel.max(), np.quantile(rel, 0.99), hit.sum()))
    assert agree.mean() >= 0.995 and hit.sum() > 1000
    assert rel.max() <= RATIO_TOL, rel.max()
    assert abs(g["spectrum"].sum() / f["spectrum"].sum() - 1) <= SPEC_TOL
    s = ora.scene(**oracle_kwargs(cam))
    al, be = R.pixel_centres(R.camera_desc(**cam))
    rows, cols = np.nonzero(hit)
    for q in np.random.default_rng(78).choice(len(rows), 12, replace=False):
        i, j = rows[q], cols[q]
        d = ora.disk_ray(s, al[j], be[i], **DISK)
        assert d["status"] == ora.DISK_HIT and d["order"] == g["order"][i, j]
        assert abs(g["ratio"][i, j] / d["ratio"] - 1) <= RATIO_TOL
