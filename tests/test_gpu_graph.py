"""CUDA-graph replay of repeated renders (raptor_graph_config): the replayed launch sequence
gives the same images and fluxes, bit for bit, as direct launches, for the FP64 path, the
mixed path (both streams) and the learned path; a slow-light batch of frames with new frame
times replays the captured graph with the new times.  Needs a GPU."""
import numpy as np
import pytest

from helpers import grid_plasma_kwargs
from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


def _ctx(R, prec, flags=0, graphs=True):
    cam = dict(scenes.SMALL, nx=40, ny=32, precision=prec, flags=flags)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    ctx.graph_config(graphs)
    return ctx


@pytest.mark.parametrize("kind", ["fp64", "mixed_df", "mlp"])
def test_graph_replay_matches_direct_launches(R, kind):
    import torch

    prec, flags = {"fp64": (R.FP64, 0), "mixed_df": (R.MIXED, R.FLAG_INNER_DF64), "mlp": (R.MIXED_MLP, 0)}[kind]
    freqs = [1e10, 230e9]
    params = None
    if prec == R.MIXED_MLP:
        c0 = R.Context(R.camera_desc(**scenes.SMALL))
        x, y = c0.surrogate_generate(20000, seed=3)
        c0.surrogate_init(y, seed=4)
        c0.surrogate_train(x, y, 50, lr=1e-3, lr_final=1e-4, seed=5)
        params = c0.surrogate_get()
    direct = _ctx(R, prec, flags, graphs=False)
    graph = _ctx(R, prec, flags, graphs=True)
    for c in (direct, graph):
        if params is not None:
            c.surrogate_set(params)
    ref, fref = direct.render(freqs)
    ref = ref.cpu().numpy()
    out = torch.empty((len(freqs), 32, 40), dtype=torch.float64, device="cuda")
    graph.render(freqs, image=out)  # first render: allocates the context's buffers (a new epoch)
    assert graph.graph_stats() == (0, 0)
    for call in range(4):
        out.fill_(-1.0)
        _, fl = graph.render(freqs, image=out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref), call
        assert np.array_equal(fl, fref), call
    captures, replays = graph.graph_stats()
    assert captures == 1 and replays == 3
    # another camera time (a different launch): runs directly, then is captured anew
    graph.render(freqs, image=out, t_obs=5.0)
    assert graph.graph_stats() == (1, 3)
    assert direct.graph_stats() == (0, 0)


def test_lightcurve_batch_replays_with_new_frame_times(R):
    """Slow light: the frame times live in a context buffer, so the second batch's graph is
    replayed by the third batch with other times; every batch equals a direct light curve."""
    fields, meta = scenes.torus_snapshots(6, dt_snap=10.0, n1=32, n2=32, n_modes=64, seed=scenes.SLOW["seed"])
    cam = dict(scenes.SMALL, spin=scenes.TORUS["spin"], nx=20, ny=16)  # 3 frames: under the graph size limit

    def make(graphs):
        ctx = R.Context(R.camera_desc(**cam))
        ctx.load_plasma(R.plasma_desc(**grid_plasma_kwargs(meta, scenes.DISK_MODEL, 1, -30.0)), fields=fields)
        ctx.graph_config(graphs)
        return ctx

    direct, graph = make(False), make(True)
    freqs = [230e9]
    graph.lightcurve(freqs, np.array([0.0, 5.0, 10.0]))  # allocates the context's buffers
    for batch, t in enumerate([[0.0, 5.0, 10.0], [0.0, 5.0, 10.0], [2.0, 7.0, 21.0]]):
        fl_g = graph.lightcurve(freqs, np.array(t))
        fl_d = direct.lightcurve(freqs, np.array(t))
        assert np.array_equal(fl_g, fl_d), batch
    assert graph.graph_stats() == (1, 2)


def test_large_calls_run_directly(R):
    """Calls beyond 2^19 rays launch directly (no capture)."""
    import torch

    cam = dict(scenes.SMALL, nx=1024, ny=520, precision=R.MIXED, flags=R.FLAG_INNER_DF64)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    out = torch.empty((1, 520, 1024), dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.render([230e9], image=out, flux=False)
    torch.cuda.synchronize()
    assert ctx.graph_stats() == (0, 0)
