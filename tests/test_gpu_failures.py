"""Failure handling, exercised without any device fault: a tensor-core wait that ran out is
reported and the context recovers (the flag is set from the host), and corrupt snapshot
cells (NaN velocities, negative or NaN densities, a NaN internal energy, an infinite field,
written into the arrays on the host) act as empty space: no ray ends in error, the image
and the flux stay finite and equal the oracle's on the same arrays.  Needs a GPU."""
import numpy as np
import pytest

from helpers import grid_oracle_scene, grid_plasma_kwargs, rel_err
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


def test_tensor_core_wait_timeout_reported_then_recovered(R):
    """A bounded tensor-core wait that runs out leaves its flag set: the next synchronising
    learned render returns RAPTOR_ETIMEOUT with the reason in raptor_last_error, and the
    render after it succeeds with the same image as before the fault."""
    import torch

    cam = dict(scenes.SMALL, nx=32, ny=24)
    ctx = R.Context(R.camera_desc(**cam, precision=R.MIXED_MLP, flags=R.FLAG_INNER_DF64))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    x, y = ctx.surrogate_generate(8192, seed=3)
    ctx.surrogate_init(y, seed=4)
    ctx.surrogate_train(x, y, 50, seed=5)
    freqs = [230e9]
    img0, fl0 = ctx.render(freqs)
    torch.cuda.synchronize()
    ref = img0.cpu().numpy().copy()
    ctx.inject_fault(R.FAULT_TC_WAIT)
    with pytest.raises(R.RaptorError) as ei:
        ctx.render(freqs)
    assert ei.value.status == R.ETIMEOUT
    assert "tensor-core wait" in str(ei.value)
    img1, fl1 = ctx.render(freqs)
    torch.cuda.synchronize()
    assert np.array_equal(img1.cpu().numpy(), ref)
    assert fl1[0] == fl0[0]
    # a context without a network has nothing to time out
    plain = R.Context(R.camera_desc(**cam))
    with pytest.raises(R.RaptorError) as e2:
        plain.inject_fault(R.FAULT_TC_WAIT)
    assert e2.value.status == R.EUNSUPPORTED
    with pytest.raises(R.RaptorError) as e3:
        ctx.inject_fault(99)
    assert e3.value.status == R.EINVAL


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_corrupt_snapshot_cells(R, ora, prec):
    """Snapshot cells with NaN velocities, negative or NaN densities, a NaN internal energy or
    an infinite field strength (written into the arrays on the host) emit and absorb nothing:
    a sample whose interpolated primitives are not a valid plasma state (rho <= 0, u <= 0, or
    b.b not positive, which NaN and infinite inputs make it) is treated as empty space, on
    both sides.  No ray ends in error, the error counter agrees with the status image, the
    image and the flux stay finite, the corrupted cells change the flux, and on the FP64
    path every pixel and status equals the oracle's on the same corrupted arrays."""
    import torch

    fields, meta = scenes.torus_snapshots(1, n1=64, n2=64, n_modes=128)
    bad = np.array(fields, copy=True)
    n2 = meta["n2"]
    # NaN velocities in the torus body near the equator (r ~ 6.6-9 M)
    bad[0, 2:5, n2 // 2 - 3:n2 // 2 + 3, 28:34] = np.nan
    # negative and NaN densities, a NaN internal energy and an infinite field elsewhere in it
    bad[0, 0, n2 // 2 - 8:n2 // 2 - 4, 20:26] = -1.0
    bad[0, 0, n2 // 2 + 4:n2 // 2 + 8, 36:40] = np.nan
    bad[0, 1, n2 // 2 + 10:n2 // 2 + 12, 22:30] = np.nan
    bad[0, 6, n2 // 2 - 12:n2 // 2 - 9, 30:36] = np.inf
    cam = dict(scenes.SMALL, spin=scenes.TORUS["spin"], nx=48, ny=40)
    freqs = [230e9]
    model = scenes.DISK_MODEL
    precision = R.FP64 if prec == "fp64" else R.MIXED

    def run(arr):
        ctx = R.Context(R.camera_desc(**cam, precision=precision))
        ctx.load_plasma(R.plasma_desc(**grid_plasma_kwargs(meta, model)), fields=arr)
        ctx.stats_reset()
        steps = torch.zeros((cam["ny"], cam["nx"]), dtype=torch.int32, device="cuda")
        status = torch.zeros_like(steps)
        img, fl = ctx.render(freqs, steps=steps, status=status)
        torch.cuda.synchronize()
        return img.cpu().numpy(), fl, status.cpu().numpy(), ctx.stats(), ctx.cam.t_delay

    img, fl, status, st, t_delay = run(bad)
    assert st["errors"] == int((status == R.RAY_ERROR).sum()) == 0
    assert np.all(np.isfinite(img)) and np.all(np.isfinite(fl)) and fl[0] > 0
    clean_img, clean_fl, _, _, _ = run(fields)
    assert abs(fl[0] / clean_fl[0] - 1) > 1e-3
    s = grid_oracle_scene(ora, cam, bad, meta, model)
    oimg, _, ostat = ora.render(s, freqs, t_cam=t_delay)
    assert np.all(np.isfinite(oimg))
    if prec == "fp64":
        assert np.array_equal(status, ostat)
        assert rel_err(img[0], oimg[0]).max() <= 1e-8
        assert abs(fl[0] / oimg[0].sum() - 1) <= 1e-10
    else:
        assert abs(fl[0] / oimg[0].sum() - 1) <= 1e-3
