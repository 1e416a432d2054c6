"""B300-native backward Kerr ray tracing with synchrotron radiative transfer.

Thin ctypes binding over ``libraptor.so`` (the C ABI of ``include/raptor.h``).  Every step
of the computation runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch supplies device memory and streams.  Importing works without a GPU,
but every call that needs the library fails loudly if ``libraptor.so`` is missing.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libraptor.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOPLASMA, EUNSUPPORTED = range(7)
FP64, MIXED, MIXED_MLP = 0, 1, 2
PLASMA_ANALYTIC, PLASMA_GRID = 0, 1
FLAG_K2_EXACT, FLAG_STEP_LINEAR_R, FLAG_INNER_DF64, FLAG_VERLET, FLAG_VERLET_REEVAL = 0x1, 0x2, 0x4, 0x8, 0x10
FLAG_FORWARD_RT = 0x20
MLP_TCGEN05, MLP_MMA_SYNC = 0, 1
FAULT_TC_WAIT = 1
RAY_ESCAPED, RAY_CAPTURED, RAY_THICK, RAY_TRUNCATED, RAY_ERROR = range(5)

EXPORTS = [
    "raptor_version", "raptor_camera_desc_default", "raptor_plasma_desc_default", "raptor_camera_init",
    "raptor_camera_set", "raptor_load_plasma", "raptor_render", "raptor_render_ex", "raptor_render_host",
    "raptor_lightcurve", "raptor_trace_ray", "raptor_stats", "raptor_stats_reset", "raptor_stats_ex", "raptor_set_launch",
    "raptor_last_error", "raptor_destroy", "raptor_profile", "raptor_profile_read", "raptor_measure_fma_peak",
    "raptor_render_noalloc", "raptor_autotune", "raptor_surrogate_param_count", "raptor_surrogate_generate",
    "raptor_surrogate_init", "raptor_surrogate_train", "raptor_surrogate_grad", "raptor_surrogate_eval",
    "raptor_surrogate_get", "raptor_surrogate_set", "raptor_surrogate_save", "raptor_surrogate_load", "raptor_surrogate_config", "raptor_surrogate_kernel",
    "raptor_disk_desc_default", "raptor_disk_render", "raptor_disk_render_learned", "raptor_crossings_param_count",
    "raptor_crossings_generate", "raptor_crossings_init", "raptor_crossings_train", "raptor_crossings_grad",
    "raptor_crossings_eval", "raptor_crossings_get", "raptor_crossings_set", "raptor_crossings_config", "raptor_mixed_config", "raptor_long_config", "raptor_profile_timeline", "raptor_graph_config", "raptor_graph_stats", "raptor_check_fp32_math",
    "raptor_inject_fault", "raptor_crossings_confidence", "raptor_surrogate_handoff",
]
KERNEL_NAMES = ["render_fp64", "mixed_fp32_in", "mixed_fp64", "mixed_fp32_out", "reduce", "trace", "load", "peak",
                "surrogate", "train", "surrogate_mlp", "disk", "mixed_fp64_long"]


class RaptorError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"raptor status {status}: {msg}")
        self.status = status


class CameraDesc(C.Structure):
    _fields_ = [
        ("spin", C.c_double), ("mass_msun", C.c_double), ("distance_pc", C.c_double),
        ("r_cam", C.c_double), ("incl_deg", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
        ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("beta_min", C.c_double), ("beta_max", C.c_double),
        ("eps", C.c_double), ("r_stop_factor", C.c_double), ("r_escape", C.c_double), ("tau_cut", C.c_double),
        ("max_steps", C.c_int), ("precision", C.c_int), ("flags", C.c_uint), ("reserved0", C.c_int),
        ("r_fp64", C.c_double), ("turn_kr", C.c_double), ("t_delay", C.c_double),
    ]


class DiskDesc(C.Structure):
    _fields_ = [
        ("r_in", C.c_double), ("r_out", C.c_double), ("q", C.c_double), ("max_cross", C.c_int),
        ("profile_order", C.c_int), ("n_bins", C.c_int), ("x_min", C.c_double), ("x_max", C.c_double),
    ]


class PlasmaDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("slow_light", C.c_int),
        ("n0", C.c_double), ("n_pow", C.c_double), ("the0", C.c_double), ("the_pow", C.c_double),
        ("B0_gauss", C.c_double), ("B_pow", C.c_double),
        ("fields", C.c_void_p), ("n1", C.c_int), ("n2", C.c_int), ("n_snap", C.c_int), ("fields_on_device", C.c_int),
        ("x1_min", C.c_double), ("x1_max", C.c_double), ("h_mks", C.c_double),
        ("t0", C.c_double), ("dt_snap", C.c_double), ("mass_unit_g", C.c_double),
        ("r_high", C.c_double), ("r_low", C.c_double), ("gamma_ad", C.c_double), ("theta_e_min", C.c_double),
    ]


_lib = None


def lib():
    """Load libraptor.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1801_10452_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, ip, dp, st = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int
        u64p = C.POINTER(C.c_ulonglong)
        sig = {
            "raptor_version": (C.c_int, []),
            "raptor_camera_desc_default": (None, [C.POINTER(CameraDesc)]),
            "raptor_plasma_desc_default": (None, [C.POINTER(PlasmaDesc)]),
            "raptor_camera_init": (st, [C.POINTER(CameraDesc), C.POINTER(vp)]),
            "raptor_camera_set": (st, [vp, C.POINTER(CameraDesc)]),
            "raptor_load_plasma": (st, [vp, C.POINTER(PlasmaDesc), vp]),
            "raptor_render": (st, [vp, dp, C.c_int, C.c_double, vp, dp, vp]),
            "raptor_render_ex": (st, [vp, dp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, vp, dp, vp, vp, vp]),
            "raptor_render_host": (st, [vp, dp, C.c_int, C.c_double, dp, dp, vp]),
            "raptor_lightcurve": (st, [vp, dp, C.c_int, dp, C.c_int, C.c_int, dp, vp, vp]),
            "raptor_trace_ray": (st, [vp, C.c_double, C.c_double, C.c_double, dp, C.c_int, C.c_int, dp, ip, ip, dp, vp]),
            "raptor_stats": (st, [vp, u64p, u64p, u64p, u64p, u64p, u64p]),
            "raptor_stats_reset": (st, [vp]),
            "raptor_stats_ex": (st, [vp, vp, C.c_int]),
            "raptor_set_launch": (st, [vp, C.c_int, C.c_int, C.c_int]),
            "raptor_last_error": (C.c_char_p, [vp]),
            "raptor_destroy": (None, [vp]),
            "raptor_profile": (st, [vp, C.c_int]),
            "raptor_profile_read": (st, [vp, dp, C.POINTER(C.c_longlong)]),
            "raptor_measure_fma_peak": (st, [C.c_int, dp]),
            "raptor_autotune": (st, [vp, dp, C.c_int, C.c_double, ip, ip, ip, dp, vp]),
            "raptor_surrogate_param_count": (C.c_int, []),
            "raptor_surrogate_generate": (st, [vp, C.c_longlong, C.c_ulonglong, C.c_double, C.c_double, C.c_double,
                                               C.c_double, vp, vp, vp, vp]),
            "raptor_surrogate_init": (st, [vp, vp, C.c_longlong, C.c_ulonglong, vp]),
            "raptor_surrogate_train": (st, [vp, vp, vp, C.c_longlong, C.c_int, C.c_double, C.c_double, C.c_ulonglong, dp, vp]),
            "raptor_surrogate_grad": (st, [vp, vp, vp, C.c_longlong, C.POINTER(C.c_float), dp, vp]),
            "raptor_surrogate_eval": (st, [vp, vp, C.c_longlong, vp, vp]),
            "raptor_surrogate_get": (st, [vp, C.POINTER(C.c_float), C.c_int]),
            "raptor_surrogate_set": (st, [vp, C.POINTER(C.c_float), C.c_int]),
            "raptor_surrogate_save": (st, [vp, C.c_char_p]),
            "raptor_surrogate_load": (st, [vp, C.c_char_p]),
            "raptor_surrogate_config": (st, [vp, C.c_double, C.c_double]),
            "raptor_inject_fault": (st, [vp, C.c_int]),
            "raptor_surrogate_handoff": (st, [vp, C.c_int]),
            "raptor_crossings_confidence": (st, [vp, C.c_double, C.c_double]),
            "raptor_surrogate_kernel": (st, [vp, C.c_int]),
            "raptor_crossings_param_count": (C.c_int, []),
            "raptor_crossings_generate": (st, [vp, C.c_longlong, C.c_ulonglong, C.c_double, C.c_double, C.c_double,
                                               C.c_double, vp, vp, vp, vp]),
            "raptor_crossings_init": (st, [vp, vp, vp, C.c_longlong, C.c_ulonglong, vp]),
            "raptor_crossings_train": (st, [vp, vp, vp, C.c_longlong, C.c_int, C.c_double, C.c_double, C.c_ulonglong, dp, vp]),
            "raptor_crossings_grad": (st, [vp, vp, vp, C.c_longlong, C.POINTER(C.c_float), dp, vp]),
            "raptor_crossings_eval": (st, [vp, vp, C.c_longlong, vp, vp]),
            "raptor_crossings_get": (st, [vp, C.POINTER(C.c_float), C.c_int]),
            "raptor_crossings_set": (st, [vp, C.POINTER(C.c_float), C.c_int]),
            "raptor_crossings_config": (st, [vp, C.c_double, C.c_int]),
            "raptor_mixed_config": (st, [vp, C.c_double, C.c_int, C.c_void_p, C.c_int]),
            "raptor_long_config": (st, [vp, C.c_int, C.c_int, C.c_void_p]),
            "raptor_profile_timeline": (st, [vp, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.POINTER(C.c_int)]),
            "raptor_graph_config": (st, [vp, C.c_int]),
            "raptor_check_fp32_math": (st, [C.c_longlong, C.c_void_p]),
            "raptor_graph_stats": (st, [vp, C.c_void_p, C.c_void_p]),
            "raptor_render_noalloc": (st, [C.POINTER(CameraDesc), C.POINTER(PlasmaDesc), dp, C.c_int, C.c_double, vp, vp, vp]),
            "raptor_disk_desc_default": (st, [C.POINTER(DiskDesc)]),
            "raptor_disk_render": (st, [vp, C.POINTER(DiskDesc), vp, vp, vp, vp, vp, dp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def camera_desc(**kw) -> CameraDesc:
    d = CameraDesc()
    lib().raptor_camera_desc_default(C.byref(d))
    for k, v in kw.items():
        if not hasattr(d, k):
            raise AttributeError(k)
        setattr(d, k, v)
    return d


def plasma_desc(**kw) -> PlasmaDesc:
    d = PlasmaDesc()
    lib().raptor_plasma_desc_default(C.byref(d))
    for k, v in kw.items():
        if k == "fields":
            continue
        if not hasattr(d, k):
            raise AttributeError(k)
        setattr(d, k, v)
    return d


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _freqs(freqs):
    return np.ascontiguousarray(np.atleast_1d(np.asarray(freqs, dtype=np.float64)))


def _stream(stream):
    if stream is None:
        import torch

        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def pinned_host_array(shape):
    """A float64 host array in page-locked memory (for render_host's `out`): device-to-host
    copies into it run as direct DMA instead of through a staging buffer."""
    import torch

    return torch.empty(tuple(shape), dtype=torch.float64, pin_memory=True).numpy()


class Context:
    """One camera (sec. 2.3) with its device work buffers."""

    def __init__(self, cam: CameraDesc | None = None, **kw):
        self.cam = cam if cam is not None else camera_desc(**kw)
        h = C.c_void_p()
        st = lib().raptor_camera_init(C.byref(self.cam), C.byref(h))
        if st != OK:
            raise RaptorError(st, "raptor_camera_init rejected the camera descriptor")
        self._h = h
        self._keep = None

    def _check(self, st, what):
        if st != OK:
            msg = lib().raptor_last_error(self._h)
            raise RaptorError(st, f"{what}: {msg.decode() if msg else ''}")

    @property
    def handle(self):
        return self._h

    def set_camera(self, cam: CameraDesc | None = None, **kw):
        if cam is None:
            cam = self.cam
            for k, v in kw.items():
                setattr(cam, k, v)
        self._check(lib().raptor_camera_set(self._h, C.byref(cam)), "raptor_camera_set")
        self.cam = cam

    def load_plasma(self, desc: PlasmaDesc | None = None, fields=None, stream=None, **kw):
        """Analytic plasma (default) or a grid: `fields` is a float32 array/tensor
        [n_snap][8][n2][n1] on the host (numpy) or the device (torch)."""
        if desc is None:
            desc = plasma_desc(**kw)
        if fields is not None:
            if isinstance(fields, np.ndarray):
                f = np.ascontiguousarray(fields, dtype=np.float32)
                desc.fields = f.ctypes.data
                desc.fields_on_device = 0
            else:
                import torch

                f = fields.contiguous().to(torch.float32)
                desc.fields = f.data_ptr()
                desc.fields_on_device = 1 if f.is_cuda else 0
            desc.n_snap, _, desc.n2, desc.n1 = f.shape
            desc.kind = PLASMA_GRID
            self._keep = f
        self._check(lib().raptor_load_plasma(self._h, C.byref(desc), _stream(stream)), "raptor_load_plasma")
        self.plasma = desc
        return self

    def render(self, freqs, t_obs=0.0, image=None, stream=None, flux=True, row0=0, n_rows=None, snap=0,
               steps=None, status=None):
        """Render into `image` (torch float64 cuda [n_freq][n_rows][nx]; allocated if None).
        Returns (image, flux_jy numpy [n_freq] or None)."""
        import torch

        nu = _freqs(freqs)
        n_rows = self.cam.ny if n_rows is None else n_rows
        if image is None:
            image = torch.empty((nu.size, n_rows, self.cam.nx), dtype=torch.float64, device="cuda")
        fl = np.zeros(nu.size) if flux else None
        st = lib().raptor_render_ex(
            self._h, _dp(nu), nu.size, float(t_obs), int(row0), int(n_rows), int(snap), C.c_void_p(image.data_ptr()),
            _dp(fl) if flux else None, C.c_void_p(steps.data_ptr()) if steps is not None else None,
            C.c_void_p(status.data_ptr()) if status is not None else None, _stream(stream))
        self._check(st, "raptor_render_ex")
        return image, fl

    def render_host(self, freqs, t_obs=0.0, want_image=True, stream=None, out=None):
        """Render into host memory: (image, flux).  `out`, if given, is a C-contiguous float64
        host array of shape (n_freq, ny, nx) that receives the image (page-locked memory from
        pinned_host_array makes the copy a direct DMA); otherwise a new array is returned."""
        nu = _freqs(freqs)
        if out is not None:
            shape = (nu.size, self.cam.ny, self.cam.nx)
            if out.dtype != np.float64 or tuple(out.shape) != shape or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a C-contiguous float64 array of shape %s" % (shape,))
            img = out
        else:
            img = np.zeros((nu.size, self.cam.ny, self.cam.nx)) if want_image else None
        fl = np.zeros(nu.size)
        st = lib().raptor_render_host(self._h, _dp(nu), nu.size, float(t_obs), _dp(img) if want_image else None, _dp(fl),
                                      _stream(stream))
        self._check(st, "raptor_render_host")
        return img, fl

    def lightcurve(self, freqs, t_obs, first_frame=0, images=None, stream=None):
        nu = _freqs(freqs)
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(t_obs, dtype=np.float64)))
        fl = np.zeros((t.size, nu.size))
        st = lib().raptor_lightcurve(self._h, _dp(nu), nu.size, _dp(t), t.size, int(first_frame), _dp(fl),
                                     C.c_void_p(images.data_ptr()) if images is not None else None, _stream(stream))
        self._check(st, "raptor_lightcurve")
        return fl

    def trace_ray(self, alpha, beta, freqs, t_obs=0.0, max_rec=20000, stream=None):
        nu = _freqs(freqs)
        rec = np.zeros((max(max_rec, 1), 12))
        n = C.c_int(0)
        s = C.c_int(0)
        Iv = np.zeros(nu.size)
        st = lib().raptor_trace_ray(self._h, float(alpha), float(beta), float(t_obs), _dp(nu), nu.size, int(max_rec),
                                    _dp(rec), C.byref(n), C.byref(s), _dp(Iv), _stream(stream))
        self._check(st, "raptor_trace_ray")
        return dict(steps=n.value, status=s.value, I=Iv, trace=rec[: min(n.value, max_rec)].copy())

    def stats(self):
        v = [C.c_ulonglong(0) for _ in range(6)]
        self._check(lib().raptor_stats(self._h, *[C.byref(x) for x in v]), "raptor_stats")
        return dict(zip(["rays", "steps", "fp64_steps", "truncated", "errors", "fallback"], [x.value for x in v]))

    def stats_ex(self):
        """All counters: rays, steps, fp64_steps, truncated, errors, fallback, reentries,
        clamped, fp64_steps_long (second stream), fp32_steps_in / fp32_steps_out (FP32 steps
        executed by the mixed path's inbound and outbound phases)."""
        v = (C.c_ulonglong * 11)()
        self._check(lib().raptor_stats_ex(self._h, v, 11), "raptor_stats_ex")
        return dict(zip(["rays", "steps", "fp64_steps", "truncated", "errors", "fallback", "reentries", "clamped",
                         "fp64_steps_long", "fp32_steps_in", "fp32_steps_out"], [int(x) for x in v]))

    def stats_reset(self):
        self._check(lib().raptor_stats_reset(self._h), "raptor_stats_reset")

    def set_launch(self, threads_per_block, blocks_per_sm, blocks_per_sm_fp64=2):
        self._check(lib().raptor_set_launch(self._h, int(threads_per_block), int(blocks_per_sm), int(blocks_per_sm_fp64)),
                    "raptor_set_launch")

    def autotune(self, freqs, t_obs=0.0, stream=None):
        """Choose the fastest launch shape for this camera; returns it with its time."""
        nu = _freqs(freqs)
        tb, bps, b64 = C.c_int(0), C.c_int(0), C.c_int(0)
        ms = C.c_double(0.0)
        self._check(lib().raptor_autotune(self._h, _dp(nu), nu.size, float(t_obs), C.byref(tb), C.byref(bps), C.byref(b64),
                                          C.byref(ms), _stream(stream)), "raptor_autotune")
        return dict(threads_per_block=tb.value, blocks_per_sm=bps.value, blocks_per_sm_fp64=b64.value, ms=ms.value)

    def profile(self, enable=True):
        self._check(lib().raptor_profile(self._h, 1 if enable else 0), "raptor_profile")

    def profile_read(self):
        """{kernel name: (ms, launches)} since the last profile(True)."""
        k = len(KERNEL_NAMES)
        ms = np.zeros(k)
        n = (C.c_longlong * k)()
        self._check(lib().raptor_profile_read(self._h, _dp(ms), n), "raptor_profile_read")
        return {KERNEL_NAMES[i]: (float(ms[i]), int(n[i])) for i in range(k)}

    def disk_render(self, r_in=0.0, r_out=15.0, q=2.0, max_cross=10, profile_order=1, n_bins=64, x_range=(0.2, 1.6),
                    spectrum=True, stream=None, learned=False):
        """Thin-disk line emitter (sec. 4.2.1) with this context's camera, in FP64: per pixel
        E_obs/E_em, line intensity and hit order (device tensors [ny][nx]), status and steps,
        and the line spectrum (host array [n_bins], None without `spectrum`) with its bin
        edges.  `learned`: from the crossing network outside the critical curve's fallback
        band (raptor_disk_render_learned)."""
        import torch

        d = DiskDesc()
        lib().raptor_disk_desc_default(C.byref(d))
        d.r_in, d.r_out, d.q, d.max_cross = float(r_in), float(r_out), float(q), int(max_cross)
        d.profile_order, d.n_bins, d.x_min, d.x_max = int(profile_order), int(n_bins), float(x_range[0]), float(x_range[1])
        shape = (self.cam.ny, self.cam.nx)
        ratio = torch.empty(shape, dtype=torch.float64, device="cuda")
        inten = torch.empty_like(ratio)
        order = torch.empty(shape, dtype=torch.int32, device="cuda")
        status = torch.empty_like(order)
        steps = torch.empty_like(order)
        prof = np.zeros(max(1, n_bins)) if spectrum else None
        fn = "raptor_disk_render_learned" if learned else "raptor_disk_render"
        self._check(getattr(lib(), fn)(self._h, C.byref(d), C.c_void_p(ratio.data_ptr()), C.c_void_p(inten.data_ptr()),
                                       C.c_void_p(order.data_ptr()), C.c_void_p(status.data_ptr()),
                                       C.c_void_p(steps.data_ptr()), _dp(prof) if spectrum else None, _stream(stream)), fn)
        edges = np.linspace(x_range[0], x_range[1], n_bins + 1)
        return dict(ratio=ratio, intensity=inten, order=order, status=status, steps=steps,
                    spectrum=prof[:n_bins] if spectrum else None, edges=edges)

    def profile_timeline(self):
        """Recorded launches since the last profile(True), in launch order: a list of
        (kernel name, lane, start ms, duration ms); lane 1 is the mixed path's second stream."""
        n = C.c_int(0)
        self._check(lib().raptor_profile_timeline(self._h, 0, None, None, None, None, C.byref(n)),
                    "raptor_profile_timeline")
        k = n.value
        slot = np.zeros(k, dtype=np.int32)
        lane = np.zeros(k, dtype=np.int32)
        t0 = np.zeros(k)
        dt = np.zeros(k)
        if k:
            self._check(lib().raptor_profile_timeline(self._h, k, _ip(slot), _ip(lane), _dp(t0), _dp(dt), C.byref(n)),
                        "raptor_profile_timeline")
        return [(KERNEL_NAMES[slot[i]], int(lane[i]), float(t0[i]), float(dt[i])) for i in range(k)]

    # ---- learned surrogate -------------------------------------------------------------
    def surrogate_generate(self, n, seed=0x1801104520000005, spin=(0.0, 0.99), incl=(5.0, 85.0), states=False,
                           stream=None):
        """Integrator-generated training set: (inputs float32 [n][4], targets float64 [n][6]
        [, raw states float64 [n][6]])."""
        import torch

        x = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        y = torch.empty((n, 6), dtype=torch.float64, device="cuda")
        z = torch.empty((n, 6), dtype=torch.float64, device="cuda") if states else None
        self._check(lib().raptor_surrogate_generate(self._h, int(n), int(seed), float(spin[0]), float(spin[1]), float(incl[0]),
                                                    float(incl[1]), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                    C.c_void_p(z.data_ptr()) if states else None, _stream(stream)),
                    "raptor_surrogate_generate")
        return (x, y, z) if states else (x, y)

    def surrogate_init(self, targets, seed=7, stream=None):
        self._check(lib().raptor_surrogate_init(self._h, C.c_void_p(targets.data_ptr()), int(targets.shape[0]), int(seed),
                                                _stream(stream)), "raptor_surrogate_init")

    def surrogate_train(self, inputs, targets, steps, lr=2e-3, lr_final=2e-5, seed=11, record_loss=False, stream=None):
        loss = np.zeros(steps) if record_loss else None
        self._check(lib().raptor_surrogate_train(self._h, C.c_void_p(inputs.data_ptr()), C.c_void_p(targets.data_ptr()),
                                                 int(inputs.shape[0]), int(steps), float(lr), float(lr_final), int(seed),
                                                 _dp(loss) if record_loss else None, _stream(stream)), "raptor_surrogate_train")
        return loss

    def surrogate_grad(self, inputs, targets, stream=None):
        n = lib().raptor_surrogate_param_count() - 24
        g = np.zeros(n, dtype=np.float32)
        L = C.c_double(0.0)
        self._check(lib().raptor_surrogate_grad(self._h, C.c_void_p(inputs.data_ptr()), C.c_void_p(targets.data_ptr()),
                                                int(inputs.shape[0]), g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(L),
                                                _stream(stream)), "raptor_surrogate_grad")
        return g, L.value

    def surrogate_eval(self, inputs, stream=None):
        import torch

        pred = torch.empty((inputs.shape[0], 6), dtype=torch.float64, device="cuda")
        self._check(lib().raptor_surrogate_eval(self._h, C.c_void_p(inputs.data_ptr()), int(inputs.shape[0]),
                                                C.c_void_p(pred.data_ptr()), _stream(stream)), "raptor_surrogate_eval")
        return pred

    def surrogate_get(self):
        n = lib().raptor_surrogate_param_count()
        P = np.zeros(n, dtype=np.float32)
        self._check(lib().raptor_surrogate_get(self._h, P.ctypes.data_as(C.POINTER(C.c_float)), n), "raptor_surrogate_get")
        return P

    def surrogate_set(self, P):
        P = np.ascontiguousarray(P, dtype=np.float32)
        self._check(lib().raptor_surrogate_set(self._h, P.ctypes.data_as(C.POINTER(C.c_float)), P.size), "raptor_surrogate_set")

    # ---- crossing network (the surrogate's equatorial outputs) ---------------------------
    def crossings_generate(self, n, seed=0x1801104520000005, spin=(0.0, 0.99), incl=(5.0, 85.0), raw=False,
                           stream=None):
        """Integrator-generated crossing set: (inputs float32 [n][4], targets float64 [n][16]
        [, raw float64 [n][16]: per crossing presence, r, lambda, E_obs/E_em])."""
        import torch

        x = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        y = torch.empty((n, 16), dtype=torch.float64, device="cuda")
        z = torch.empty((n, 16), dtype=torch.float64, device="cuda") if raw else None
        self._check(lib().raptor_crossings_generate(self._h, int(n), int(seed), float(spin[0]), float(spin[1]),
                                                    float(incl[0]), float(incl[1]), C.c_void_p(x.data_ptr()),
                                                    C.c_void_p(y.data_ptr()), C.c_void_p(z.data_ptr()) if raw else None,
                                                    _stream(stream)), "raptor_crossings_generate")
        return (x, y, z) if raw else (x, y)

    def crossings_init(self, targets, seed=7, stream=None, inputs=None):
        """Initialise the crossing network; `inputs` (optional) sets the spin and inclination
        normalisation to their range."""
        self._check(lib().raptor_crossings_init(self._h, C.c_void_p(inputs.data_ptr()) if inputs is not None else None,
                                                C.c_void_p(targets.data_ptr()), int(targets.shape[0]), int(seed),
                                                _stream(stream)), "raptor_crossings_init")

    def crossings_train(self, inputs, targets, steps, lr=2e-3, lr_final=2e-5, seed=11, record_loss=False, stream=None):
        loss = np.zeros(steps) if record_loss else None
        self._check(lib().raptor_crossings_train(self._h, C.c_void_p(inputs.data_ptr()), C.c_void_p(targets.data_ptr()),
                                                 int(inputs.shape[0]), int(steps), float(lr), float(lr_final), int(seed),
                                                 _dp(loss) if record_loss else None, _stream(stream)),
                    "raptor_crossings_train")
        return loss

    def crossings_grad(self, inputs, targets, stream=None):
        """(gradient float32 [param_count - 40], loss) of one batch (a multiple of 128 rows)."""
        n = lib().raptor_crossings_param_count() - 40
        g = np.zeros(n, dtype=np.float32)
        L = C.c_double(0.0)
        self._check(lib().raptor_crossings_grad(self._h, C.c_void_p(inputs.data_ptr()), C.c_void_p(targets.data_ptr()),
                                                int(inputs.shape[0]), g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(L),
                                                _stream(stream)), "raptor_crossings_grad")
        return g, L.value

    def crossings_eval(self, inputs, stream=None):
        """Decoded predictions float64 [n][16]: per crossing presence probability, r, lambda,
        E_obs/E_em."""
        import torch

        pred = torch.empty((inputs.shape[0], 16), dtype=torch.float64, device="cuda")
        self._check(lib().raptor_crossings_eval(self._h, C.c_void_p(inputs.data_ptr()), int(inputs.shape[0]),
                                                C.c_void_p(pred.data_ptr()), _stream(stream)), "raptor_crossings_eval")
        return pred

    def crossings_get(self):
        n = lib().raptor_crossings_param_count()
        P = np.zeros(n, dtype=np.float32)
        self._check(lib().raptor_crossings_get(self._h, P.ctypes.data_as(C.POINTER(C.c_float)), n), "raptor_crossings_get")
        return P

    def crossings_set(self, P):
        P = np.ascontiguousarray(P, dtype=np.float32)
        self._check(lib().raptor_crossings_set(self._h, P.ctypes.data_as(C.POINTER(C.c_float)), P.size),
                    "raptor_crossings_set")

    def crossings_config(self, fallback_band=1.0, fallback_df64=True):
        """Fallback of the learned thin disk: band (M) around the critical curve, and whether
        its rays run in double-float arithmetic (else FP64, equal to the FP64 disk)."""
        self._check(lib().raptor_crossings_config(self._h, float(fallback_band), int(bool(fallback_df64))),
                    "raptor_crossings_config")

    def crossings_confidence(self, presence_margin=2.0, radius_margin=0.01):
        """Learned thin disk: pixels with a presence logit within presence_margin of 0, or a
        predicted radius within radius_margin (in ln r) of r_in or r_out, fall back too."""
        self._check(lib().raptor_crossings_confidence(self._h, float(presence_margin), float(radius_margin)),
                    "raptor_crossings_confidence")

    def long_config(self, threads_per_block=0, budgets=None):
        """Schedule of the near-critical rays' FP64 phase on the second stream: block size
        (0: the other launches') and the step budgets of its passes (None: one unlimited
        pass; the last pass is unlimited)."""
        b = (C.c_int * max(1, len(budgets or [])))(*[int(v) for v in (budgets or [])])
        self._check(lib().raptor_long_config(self._h, int(threads_per_block), len(budgets or []) + 1, b),
                    "raptor_long_config")

    def mixed_config(self, crit_band=0.5, budgets=None, tail_split=0):
        """Schedule of the mixed path: the near-critical band (M) whose rays run their FP64
        phase on the second stream, the step budgets of the other rays' FP64 passes (None:
        the default; the last pass is unlimited), and the number of passes after which the
        remaining FP64 work moves to the second stream (0: never)."""
        if budgets is None:
            self._check(lib().raptor_mixed_config(self._h, float(crit_band), 8, None, int(tail_split)),
                        "raptor_mixed_config")
        else:
            b = (C.c_int * max(1, len(budgets)))(*[int(v) for v in budgets])
            self._check(lib().raptor_mixed_config(self._h, float(crit_band), len(budgets) + 1, b, int(tail_split)),
                        "raptor_mixed_config")

    def graph_config(self, enable=True):
        """Replay repeated identical renders from a captured CUDA graph (default on)."""
        self._check(lib().raptor_graph_config(self._h, 1 if enable else 0), "raptor_graph_config")

    def graph_stats(self):
        """(captures, replays) of the context's render graphs."""
        c, r = C.c_longlong(0), C.c_longlong(0)
        self._check(lib().raptor_graph_stats(self._h, C.byref(c), C.byref(r)), "raptor_graph_stats")
        return int(c.value), int(r.value)

    def surrogate_kernel(self, kind):
        """Inference kernel: MLP_TCGEN05 (default) or MLP_MMA_SYNC."""
        self._check(lib().raptor_surrogate_kernel(self._h, int(kind)), "raptor_surrogate_kernel")

    def surrogate_save(self, path):
        """Write the trained network to `path` (format in raptor_surrogate_save)."""
        self._check(lib().raptor_surrogate_save(self._h, str(path).encode()), "raptor_surrogate_save")

    def surrogate_load(self, path):
        """Load a network written by surrogate_save (validated; as surrogate_set)."""
        self._check(lib().raptor_surrogate_load(self._h, str(path).encode()), "raptor_surrogate_load")

    def surrogate_handoff(self, n_steps=60):
        """Hand-off step count for the next surrogate_generate / surrogate_init (the network
        carries it; renders use the count of the network in use)."""
        self._check(lib().raptor_surrogate_handoff(self._h, int(n_steps)), "raptor_surrogate_handoff")

    def surrogate_config(self, fallback_band=0.5, r_exit=50.0):
        self._check(lib().raptor_surrogate_config(self._h, float(fallback_band), float(r_exit)), "raptor_surrogate_config")

    def inject_fault(self, kind=1):
        """Host-side fault injection (raptor_inject_fault): kind 1 sets the tensor-core wait
        flag, so that the next synchronising learned render returns RAPTOR_ETIMEOUT."""
        self._check(lib().raptor_inject_fault(self._h, int(kind)), "raptor_inject_fault")

    def close(self):
        if getattr(self, "_h", None):
            lib().raptor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def measure_fma_peak(fp64: bool) -> float:
    """Achieved FMA throughput (TFLOP/s) of the current device in FP64 or FP32."""
    v = C.c_double(0.0)
    st = lib().raptor_measure_fma_peak(1 if fp64 else 0, C.byref(v))
    if st != OK:
        raise RaptorError(st, "raptor_measure_fma_peak")
    return v.value


def pixel_centres(cam: CameraDesc):
    """(alpha[nx], beta[ny]) pixel centres of the camera (sec. 2.3 image plane)."""
    da = (cam.alpha_max - cam.alpha_min) / cam.nx
    db = (cam.beta_max - cam.beta_min) / cam.ny
    return cam.alpha_min + (np.arange(cam.nx) + 0.5) * da, cam.beta_min + (np.arange(cam.ny) + 0.5) * db


def check_fp32_math(n=1 << 24):
    """Largest ulp distances of the library's FP32 primitives from their references:
    {"rcp", "sqrt", "cbrt", "x_over_expm1", "one_minus_exp_over"}."""
    u = (C.c_uint * 5)()
    st = lib().raptor_check_fp32_math(int(n), u)
    if st != OK:
        raise RaptorError(st, "raptor_check_fp32_math")
    return dict(zip(["rcp", "sqrt", "cbrt", "x_over_expm1", "one_minus_exp_over"], [int(v) for v in u]))
