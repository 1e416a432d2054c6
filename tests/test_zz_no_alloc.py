"""raptor_render_noalloc: the rendering entry point for callers that cannot allocate device
memory (a host program whose memory pool already holds the GPU, or a path that must not
call cudaMalloc/cudaFree after start-up).  Called through the C ABI with ctypes and checked
against raptor_render on the same inputs, on two calls in a row.  Named to run last.
Needs a GPU."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PIX_TOL = 1e-8   # the FP64 parity bound of the other GPU tests
FLUX_TOL = 1e-10


def test_noalloc_render_matches_render_twice():
    import torch

    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R
    from paper_1801_10452_b300 import scenes

    L = C.CDLL(R.LIB_PATH)
    cam = R.CameraDesc()
    L.raptor_camera_desc_default(C.byref(cam))
    cam.spin, cam.nx, cam.ny, cam.precision = 0.9375, 40, 30, R.FP64
    pl = R.PlasmaDesc()
    L.raptor_plasma_desc_default(C.byref(pl))
    for k, v in scenes.ANALYTIC_PLASMA.items():
        setattr(pl, k, v)
    freqs = np.array(scenes.SPECTRAL_FREQS[:3], dtype=np.float64)
    dp = C.POINTER(C.c_double)
    fptr = freqs.ctypes.data_as(dp)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    # reference: the context-based entry point
    ctx = C.c_void_p()
    assert L.raptor_camera_init(C.byref(cam), C.byref(ctx)) == 0
    assert L.raptor_load_plasma(ctx, C.byref(pl), stream) == 0
    ref = torch.zeros((3, 30, 40), dtype=torch.float64, device="cuda")
    ref_flux = np.zeros(3)
    assert L.raptor_render(ctx, fptr, 3, C.c_double(0.0), C.c_void_p(ref.data_ptr()), ref_flux.ctypes.data_as(dp), stream) == 0
    torch.cuda.synchronize()
    ref_img = ref.cpu().numpy()
    L.raptor_destroy(ctx)

    L.raptor_render_noalloc.restype = C.c_int
    for call in range(2):
        img = torch.full((3, 30, 40), -1.0, dtype=torch.float64, device="cuda")
        flux = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = L.raptor_render_noalloc(C.byref(cam), C.byref(pl), fptr, 3, C.c_double(0.0), C.c_void_p(img.data_ptr()),
                                     C.c_void_p(flux.data_ptr()), stream)
        assert st == 0, (call, st)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call's one-time set-up, a call takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free_before
        g = img.cpu().numpy()
        fl = flux.cpu().numpy()
        den = np.maximum(np.abs(ref_img), 1e-12 * np.abs(ref_img).max())
        assert (np.abs(g - ref_img) / den).max() <= PIX_TOL, call
        assert np.all(np.abs(fl / ref_flux - 1) <= FLUX_TOL), call

    # sizes beyond the stated maximum and unsupported inputs are rejected before any launch
    many = np.full(65, 230e9)
    img = torch.zeros((65, 30, 40), dtype=torch.float64, device="cuda")
    assert L.raptor_render_noalloc(C.byref(cam), C.byref(pl), many.ctypes.data_as(dp), 65, C.c_double(0.0),
                                   C.c_void_p(img.data_ptr()), None, stream) == R.EINVAL
    cam.precision = R.MIXED
    assert L.raptor_render_noalloc(C.byref(cam), C.byref(pl), fptr, 3, C.c_double(0.0), C.c_void_p(img.data_ptr()), None,
                                   stream) == R.EINVAL
