"""Learned surrogate (RAPTOR_MIXED_MLP): integrator-generated training data against the
FP64 oracle, the library's BF16 backward pass against the FP64 network oracle, training
that generalises to held-out rays, render parity against the FP64 oracle, and the gain of the
trained network over the same path without it.  Needs a GPU."""
import time

import numpy as np
import pytest

from helpers import near_ring, oracle_kwargs, rel_err, ring_mask
from oracle import mlp
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu

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
    """A network trained on the full range of the learned workload (a in [0, 0.99],
    i in [5, 85] deg, +-20 M), shared by the render tests."""
    import torch

    ctx = R.Context(R.camera_desc(**scenes.SMALL, precision=R.MIXED_MLP))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    x, y = ctx.surrogate_generate(1_000_000, seed=5)
    ctx.surrogate_init(y, seed=7)
    loss = ctx.surrogate_train(x, y, 16000, lr=2e-3, lr_final=2e-5, seed=11)
    torch.cuda.synchronize()
    return ctx.surrogate_get()


def test_training_data_is_the_integrator_state(R, ora):
    """The generator's raw states equal the oracle's FP64 geodesic after 60 steps."""
    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    x, y, z = ctx.surrogate_generate(96, seed=3, states=True)
    xs, zs = x.cpu().numpy(), z.cpu().numpy()
    for i in range(96):
        al, be, a, inc = map(float, xs[i])
        s = ora.scene(a=a, incl_deg=inc)
        st, xf, kf, n = ora.geodesic(s, al, be, max_steps=60)
        x0, _ = ora.camera(s, al, be)
        assert n == 60
        ref = np.array([xf[0] - x0[0], np.log(xf[1]), xf[2], xf[3], kf[2], kf[1]])
        assert np.all(np.abs(zs[i] - ref) <= 1e-9 * np.maximum(np.abs(ref), 1.0)), (i, zs[i] - ref)


def test_handoff_step_count(R, ora):
    """A non-default hand-off: the generator's raw states equal the oracle's FP64 geodesic
    after that many steps, the network initialised on them carries the count in its
    parameters (read back by raptor_surrogate_set), and counts outside [1, 1000] are
    refused."""
    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    ctx.surrogate_handoff(36)
    x, y, z = ctx.surrogate_generate(32, seed=4, states=True)
    xs, zs = x.cpu().numpy(), z.cpu().numpy()
    for i in range(32):
        al, be, a, inc = map(float, xs[i])
        s = ora.scene(a=a, incl_deg=inc)
        st, xf, kf, n = ora.geodesic(s, al, be, max_steps=36)
        x0, _ = ora.camera(s, al, be)
        assert n == 36
        ref = np.array([xf[0] - x0[0], np.log(xf[1]), xf[2], xf[3], kf[2], kf[1]])
        assert np.all(np.abs(zs[i] - ref) <= 1e-9 * np.maximum(np.abs(ref), 1.0)), (i, zs[i] - ref)
    ctx.surrogate_init(y, seed=7)
    P = ctx.surrogate_get()
    assert 36.0 in P.tolist()
    for bad in (0, -3, 1001):
        with pytest.raises(R.RaptorError) as e:
            ctx.surrogate_handoff(bad)
        assert e.value.status == R.EINVAL
    other = R.Context(R.camera_desc(**scenes.SMALL, precision=R.MIXED_MLP))
    other.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    other.surrogate_set(P)
    other.render([230e9])
    Q = P.copy()
    Q[np.asarray(P) == 36.0] = 2.5   # not an integer count
    with pytest.raises(R.RaptorError) as e:
        other.surrogate_set(Q)
    assert e.value.status == R.EINVAL


def test_backward_pass_matches_fp64_oracle(R):
    """Gradient of the batch loss from the library's kernels (BF16 hidden layers, FP32
    accumulation) against the FP64 chain rule of oracle/mlp.py, per parameter tensor, at the
    initial weights (where the residuals are O(1); near convergence BF16 rounding of the
    forward pass is comparable to the residuals themselves).  Bound: 1e-2 relative L2 per
    tensor (BF16 has an 8-bit mantissa: ~4e-3 per rounding)."""
    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    x, y = ctx.surrogate_generate(4096, seed=13)
    ctx.surrogate_init(y, seed=17)
    P = ctx.surrogate_get().astype(np.float64)
    xb, yb = x[:512].contiguous(), y[:512].contiguous()
    g, L = ctx.surrogate_grad(xb, yb)
    xo, yo = xb.cpu().numpy().astype(np.float64), yb.cpu().numpy()
    go = mlp.grad(P, xo, yo)
    Lo = mlp.loss(P, xo, yo)
    assert abs(L / Lo - 1) < 2e-3
    for a, b in [(mlp.W1, mlp.B1), (mlp.B1, mlp.W2), (mlp.W2, mlp.B2), (mlp.B2, mlp.W3), (mlp.W3, mlp.B3),
                 (mlp.B3, mlp.W4), (mlp.W4, mlp.B4), (mlp.B4, mlp.NORM)]:
        e = np.linalg.norm(g[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
        assert e < 1e-2, (a, b, e)
        cos = np.dot(g[a:b], go[a:b]) / (np.linalg.norm(g[a:b]) * np.linalg.norm(go[a:b]))
        assert cos > 0.9998, (a, b, cos)


def test_training_generalises(R):
    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    x, y = ctx.surrogate_generate(300_000, seed=21)
    xh, yh = ctx.surrogate_generate(20_000, seed=22)
    ctx.surrogate_init(y, seed=23)
    loss = ctx.surrogate_train(x, y, 3000, lr=2e-3, lr_final=2e-5, seed=24, record_loss=True)
    assert np.mean(loss[-100:]) < 2e-2 * np.mean(loss[:10])
    pred = ctx.surrogate_eval(xh).cpu().numpy()
    err = np.abs(pred - yh.cpu().numpy())
    # held-out median errors of theta and ln r (the quantities the hand-off is sensitive to)
    assert np.median(err[:, 2]) < 5e-5 and np.median(err[:, 1]) < 1e-4


def _bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _forward_bf16(P, x):
    """The network in FP64 with the kernels' BF16 roundings (hidden weights, h1, h2, h3)."""
    p = mlp.unpack(P)
    xn = (x - p["shift"]) * p["scale"]
    h1 = _bf16(mlp.silu(xn @ p["W1"].T + p["b1"]))
    h2 = _bf16(mlp.silu(h1 @ _bf16(p["W2"]).T + p["b2"]))
    h3 = _bf16(mlp.silu(h2 @ _bf16(p["W3"]).T + p["b3"]))
    return h3 @ p["W4"].T + p["b4"]


@pytest.mark.parametrize("n", [1, 3001, 70000])
def test_tensor_core_inference(R, trained, n):
    """Inference on tcgen05 (default) and on mma.sync against the FP64 network with the same
    BF16 roundings, on 1 row, a ragged 23.4 tiles of 128 rows and 547 tiles (several per
    persistent CTA).  The mean error is FP32 accumulation.  An activation whose BF16 rounding
    flips by one ulp (2^-8 relative) between the FP32 and FP64 sums moves the normalised
    outputs of its row by ~1e-3 to ~1e-2 (several flips in one row: up to ~0.1); such rows
    are rare, so the 99.9th percentile stays small."""
    ctx = R.Context(R.camera_desc(**scenes.SMALL))
    ctx.surrogate_set(trained)
    P = trained.astype(np.float64)
    sd, mu = P[mlp.NORM + 16:mlp.NORM + 22], P[mlp.NORM + 8:mlp.NORM + 14]
    x, _ = ctx.surrogate_generate(n, seed=41)
    ref = _forward_bf16(P, x.cpu().numpy().astype(np.float64))[:, :6]
    outs = {}
    for kind in (R.MLP_TCGEN05, R.MLP_MMA_SYNC):
        ctx.surrogate_kernel(kind)
        outs[kind] = (ctx.surrogate_eval(x).cpu().numpy() - mu) / sd
        d = np.abs(outs[kind] - ref)
        assert d.mean() < 3e-5 and np.quantile(d, 0.999) < 5e-3 and d.max() < 0.15, (kind, d.max(), d.mean())
    assert np.abs(outs[R.MLP_TCGEN05] - outs[R.MLP_MMA_SYNC]).mean() < 3e-5
    with pytest.raises(R.RaptorError):
        ctx.surrogate_kernel(7)


def _render(R, cam, prec, freqs, params=None):
    import torch

    ctx = R.Context(R.camera_desc(**cam, precision=prec))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    if params is not None:
        ctx.surrogate_set(params)
    img, fl = ctx.render(freqs)
    torch.cuda.synchronize()
    return ctx, img.cpu().numpy(), fl


@pytest.mark.parametrize("spin", [0.9, 0.5])
def test_mixed_mlp_render_parity(R, ora, trained, spin):
    """RAPTOR_MIXED_MLP against the FP64 oracle: flux within 1e-3 and pixels outside the
    critical-curve band within 1e-2 (inside the band and the shadow the exact integrator runs)."""
    cam = dict(scenes.SMALL, spin=spin, nx=48, ny=40)
    freqs = [1e10, 230e9]
    _, img, fl = _render(R, cam, R.MIXED_MLP, freqs, trained)
    oimg, _, _ = ora.render(ora.scene(**oracle_kwargs(cam)), freqs)
    al, be = R.pixel_centres(R.camera_desc(**cam))
    band = ring_mask(al, be, spin, cam["incl_deg"], 0.5)
    for f in range(len(freqs)):
        assert abs(fl[f] / oimg[f].sum() - 1) <= FLUX_TOL
        assert rel_err(img[f], oimg[f], floor_frac=1e-6)[~band].max() <= PIX_TOL


def test_mixed_mlp_many_frequencies_ragged(R, ora, trained):
    """20 frequencies (two frequency chunks: the network's inference runs once, in the first,
    and both chunks start their rays from its states) on a ragged 37 x 29 image, with
    double-float inner steps: every frequency's flux within 1e-3 of the oracle's and every
    pixel outside the critical-curve band within 1e-2, except the pixel column on alpha = 0
    (rays through the polar axis, ill-conditioned in the method: within 0.1)."""
    cam = dict(scenes.SMALL, nx=37, ny=29)
    freqs = list(np.logspace(10, 13, 20))
    ctx = R.Context(R.camera_desc(**cam, precision=R.MIXED_MLP, flags=R.FLAG_INNER_DF64))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    ctx.surrogate_set(trained)
    img, fl = ctx.render(freqs)
    img = img.cpu().numpy()
    oimg, _, _ = ora.render(ora.scene(**oracle_kwargs(cam)), freqs)
    al, be = R.pixel_centres(R.camera_desc(**cam))
    band = ring_mask(al, be, cam["spin"], cam["incl_deg"], 0.5)
    axis = np.broadcast_to(np.abs(al)[None, :] < 1e-3, band.shape)
    assert axis.sum() == cam["ny"]
    for f in range(len(freqs)):
        assert abs(fl[f] / oimg[f].sum() - 1) <= FLUX_TOL, f
        rel = rel_err(img[f], oimg[f], floor_frac=1e-6)
        assert rel[~band & ~axis].max() <= PIX_TOL, f
        assert rel[~band & axis].max() <= 0.1, f


def test_surrogate_gain_over_the_method_without_it(R, trained):
    """What the trained network gains: the 512^2 spectral-scene image (a = 0.9375) rendered by
    the mixed path with and without the surrogate, both checked against the FP64 GPU path at
    the same 1e-3 flux bound.  The network replaces the first 60 FP32 steps of every ray it
    serves and stops outbound rays at r_exit: the FP32 phases must shrink by more than the
    surrogate stage (inputs, tensor-core network, start states) costs, in device time of each
    stage (CUDA events).  The inner FP64 phase is the same work with and without the network;
    at this size its long-ray tail dominates the frame, so the whole-frame ratio is printed,
    not bounded."""
    import torch

    cam = dict(scenes.SPECTRAL, spin=0.9375)
    freqs = [230e9]
    c64, i64, f64 = _render(R, cam, R.FP64, freqs)
    res, stages = {}, {}
    for prec in (R.MIXED, R.MIXED_MLP):
        ctx, img, fl = _render(R, cam, prec, freqs, trained if prec == R.MIXED_MLP else None)
        assert abs(fl[0] / f64[0] - 1) <= FLUX_TOL
        out = torch.empty((1, cam["ny"], cam["nx"]), dtype=torch.float64, device="cuda")
        best = 1e9
        ctx.profile(True)
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.render(freqs, image=out, flux=False)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        prof = ctx.profile_read()
        ctx.profile(False)
        res[prec] = best
        stages[prec] = {k: v[0] / 3 for k, v in prof.items() if v[1]}
    s0, s1 = stages[R.MIXED], stages[R.MIXED_MLP]
    fp32_saved = (s0["mixed_fp32_in"] + s0["mixed_fp32_out"]) - (s1["mixed_fp32_in"] + s1["mixed_fp32_out"])
    gain = res[R.MIXED] / res[R.MIXED_MLP]
    # the stage: inputs and fallback flags, the network, start states
    stage = s1["surrogate"] + s1["surrogate_mlp"]
    print(f"surrogate at 512^2: FP32 phases {fp32_saved:.2f} ms shorter, surrogate stage {stage:.2f} ms "
          f"(network {s1['surrogate_mlp']:.2f} ms); frame {gain:.3f}x (mixed {res[R.MIXED] * 1e3:.2f} ms, "
          f"mixed+MLP {res[R.MIXED_MLP] * 1e3:.2f} ms)")
    assert fp32_saved > stage


@pytest.mark.parametrize("size", [1024, 2048])
def test_learned_path_full_size(R, ora, trained, size):
    """The headline image (1024^2) and the learned-surrogate workload's render (2048^2),
    a = 0.9375, 230 GHz, through RAPTOR_MIXED_MLP with double-float inner steps, as the
    benchmark runs it: flux against the FP64 GPU path; every pixel outside the photon-ring
    band against the FP64 GPU path (itself within 1e-8 of the oracle), relative to the pixel
    for the pixels above 1e-6 of the peak and to 1e-8 of the peak below; seeded sample pixels
    and the brightest ones outside the band against the oracle tracing them one by one."""
    import torch

    cam = dict(scenes.HEADLINE, nx=size, ny=size)
    freqs = [230e9]
    ctx = R.Context(R.camera_desc(**cam, precision=R.MIXED_MLP, flags=R.FLAG_INNER_DF64))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    ctx.surrogate_set(trained)
    img, fl = ctx.render(freqs)
    c64 = R.Context(R.camera_desc(**cam, precision=R.FP64))
    c64.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    img64, f64 = c64.render(freqs)
    torch.cuda.synchronize()
    assert abs(fl[0] / f64[0] - 1) <= FLUX_TOL
    img = img.cpu().numpy()
    img64 = img64.cpu().numpy()
    al, be = R.pixel_centres(ctx.cam)
    band = _band_tree(al, be, cam)
    peak = img64[0].max()
    bright = np.abs(img64[0]) >= 1e-6 * peak
    d = np.abs(img[0] - img64[0])
    rel = d / np.maximum(np.abs(img64[0]), 1e-300)
    print(f"{size}^2 learned vs FP64 outside the band: max rel {rel[~band & bright].max():.2e} over "
          f"{int((~band & bright).sum())} pixels above 1e-6 of the peak; fainter {int((~band & ~bright).sum())} "
          f"pixels within {d[~band & ~bright].max() / peak:.1e} of the peak")
    # a pixel beyond the bound must sit on a discontinuity of the FP64 image itself (the
    # analytic flow switches from Keplerian to free fall at r_isco, so the image jumps where
    # an emitting sample crosses r_isco): there the paths disagree on an interval as wide as
    # their trajectories differ (~1e-7 M), and the FP64 image changes by more than the bound
    # within a few 1e-6 M of the pixel centre
    bad = np.argwhere(~band & bright & (rel > PIX_TOL))
    assert len(bad) <= 2, len(bad)
    for i, j in bad:
        span = 1.6e-5
        line = dict(cam, nx=16, ny=1, alpha_min=al[j] - span / 2, alpha_max=al[j] + span / 2, beta_min=be[i] - 1e-9,
                    beta_max=be[i] + 1e-9)
        cl = R.Context(R.camera_desc(**line, precision=R.FP64))
        cl.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
        v, _ = cl.render(freqs)
        v = v.cpu().numpy()[0, 0]
        print(f"pixel ({al[j]:.4f}, {be[i]:.4f}) off by {rel[i, j]:.2e}: FP64 within +-{span / 2:.0e} M spans "
              f"{v.min() / v.max():.4f} .. 1 of its largest value")
        assert v.max() / v.min() - 1 > PIX_TOL, (i, j)
    assert d[~band & ~bright].max() <= 1e-8 * peak
    s = ora.scene(**oracle_kwargs(cam))
    Lcm = ora.length_unit_cm(cam["mass_msun"])
    D = cam["distance_pc"] * 3.0856775814913673e18
    pix_jy = (al[1] - al[0]) * (be[1] - be[0]) * Lcm**2 / D**2 / 1e-23
    pix = scenes.sample_pixels(size, size, 64, seed=size)
    keep = ~band[pix[:, 0], pix[:, 1]]
    top = np.argsort(np.where(band, -np.inf, img64[0]).ravel())[-16:]
    pix = np.concatenate([pix[keep], np.stack(np.unravel_index(top, img64[0].shape), 1)])
    for (i, j) in pix:
        ov = ora.trace_ray(s, al[j], be[i], freqs)["I"][0] * pix_jy
        assert abs(img[0, i, j] - ov) <= PIX_TOL * max(abs(ov), 1e-6 * peak), (i, j)


def _band_tree(al, be, cam, width=0.5):
    """Pixels within `width` M of the critical curve, for large images (nearest vertex of a
    densely sampled curve by a k-d tree)."""
    from scipy.spatial import cKDTree

    from helpers import bardeen_critical_curve

    A, B = np.meshgrid(al, be)
    d, _ = cKDTree(bardeen_critical_curve(cam["spin"], cam["incl_deg"], 20000)).query(np.stack([A.ravel(), B.ravel()], 1))
    return (d < width).reshape(A.shape)


@pytest.mark.parametrize("fb_band", [0.5, 0.2])
def test_learned_results_independent_of_schedule(R, trained, fb_band):
    """The near-critical band only moves rays between the streams: near-critical rays are
    fallback rays (same FP32 predicate in both kernels), so whatever the band, the rays the
    network serves and every ray's arithmetic stay the same: bit-identical images and fluxes,
    also for bands wider than the fallback band."""
    import torch

    cam = dict(scenes.SMALL, nx=64, ny=56, precision=R.MIXED_MLP, flags=R.FLAG_INNER_DF64)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    ctx.surrogate_set(trained)
    ctx.surrogate_config(fb_band, 50.0)
    ctx.graph_config(False)
    freqs = [1e10, 230e9]
    ref, fref = ctx.render(freqs)
    ref = ref.cpu().numpy()
    for band in (0.0, 0.3, 0.5, 1.0, 2.0):
        ctx.mixed_config(band)
        img, fl = ctx.render(freqs)
        torch.cuda.synchronize()
        assert np.array_equal(img.cpu().numpy(), ref), band
        assert np.array_equal(fl, fref), band


def test_save_and_load_round_trip(R, trained, tmp_path):
    """A saved network loads into another context with identical parameters and renders
    identically; damaged or foreign files are refused before the context changes."""
    import torch

    cam = dict(scenes.SMALL, nx=32, ny=24, precision=R.MIXED_MLP, flags=R.FLAG_INNER_DF64)
    a = R.Context(R.camera_desc(**cam))
    a.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    a.surrogate_set(trained)
    path = tmp_path / "net.bin"
    a.surrogate_save(path)
    b = R.Context(R.camera_desc(**cam))
    b.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    with pytest.raises(R.RaptorError):
        b.surrogate_save(tmp_path / "none.bin")  # no network yet
    b.surrogate_load(path)
    assert np.array_equal(b.surrogate_get(), a.surrogate_get())
    ia, fa = a.render([230e9])
    ib, fb = b.render([230e9])
    torch.cuda.synchronize()
    assert np.array_equal(ia.cpu().numpy(), ib.cpu().numpy()) and np.array_equal(fa, fb)
    raw = path.read_bytes()
    for bad in (raw[:-1], raw + b"x", raw[:20] + bytes([raw[20] ^ 1]) + raw[21:], b"NOTAFILE" + raw[8:]):
        p = tmp_path / "bad.bin"
        p.write_bytes(bad)
        with pytest.raises(R.RaptorError):
            b.surrogate_load(p)
    assert np.array_equal(b.surrogate_get(), a.surrogate_get())
