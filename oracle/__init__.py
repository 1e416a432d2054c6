"""FP64 CPU oracle for backward Kerr ray tracing with synchrotron transfer.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product library never imports, links or calls it.

This module is a thin ctypes binding over ``raptor_oracle.cpp`` (plain C++, FP64,
``-ffp-contract=off``), which follows the paper (Bronzwaer et al. 2018, RAPTOR I) step by
step: connection from the metric (Eq. 2), RK4 (Eqs. 7-15), adaptive step (Eqs. 20-23),
camera (Eqs. 24-28), nu = -k.u (Eq. 30), backward transfer (Eqs. 34-36), Leung et al.
emissivity and Kirchhoff absorption (Eqs. 41-44), unit scaling and R-beta temperature
(Eqs. 45-46), MKS map and Newton-Raphson (App. A.2), slow light (sec. 5).

Pinned by ``tests/test_oracle_*.py`` against closed forms, invariants and the paper's
printed values.  Parity unpinned: the absolute flux of the synthetic scenes (no paper
number exists for them).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raptor_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

KIND_ANALYTIC, KIND_GRID, KIND_STATIC_ISO, KIND_BALL = 0, 1, 2, 3
ESCAPED, CAPTURED, THICK, TRUNCATED, ERROR = 0, 1, 2, 3, 4
DISK_HIT, DISK_NO_HIT = 5, 6
CROSSINGS_MAX = 7
RK4, VERLET, VERLET_REEVAL = 0, 1, 2


class OraScene(C.Structure):
    _fields_ = [
        ("m", C.c_double), ("a", C.c_double), ("coords", C.c_int), ("step_rule", C.c_int),
        ("r_cam", C.c_double), ("incl_deg", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
        ("amin", C.c_double), ("amax", C.c_double), ("bmin", C.c_double), ("bmax", C.c_double),
        ("eps", C.c_double), ("r_stop_factor", C.c_double), ("r_esc", C.c_double), ("tau_cut", C.c_double),
        ("max_steps", C.c_int), ("k2_exact", C.c_int),
        ("mass_msun", C.c_double), ("dist_pc", C.c_double),
        ("plasma_kind", C.c_int), ("slow_light", C.c_int),
        ("n0", C.c_double), ("n_pow", C.c_double), ("the0", C.c_double), ("the_pow", C.c_double),
        ("B0", C.c_double), ("B_pow", C.c_double),
        ("ball_R", C.c_double), ("ball_j", C.c_double), ("ball_alpha", C.c_double),
        ("grid", C.c_void_p), ("n1", C.c_int), ("n2", C.c_int), ("n_snap", C.c_int), ("snap", C.c_int),
        ("x1_min", C.c_double), ("x1_max", C.c_double), ("h_mks", C.c_double),
        ("t0", C.c_double), ("dt_snap", C.c_double),
        ("mass_unit_g", C.c_double), ("r_high", C.c_double), ("r_low", C.c_double), ("gamma_ad", C.c_double),
        ("integrator", C.c_int), ("theta_e_min", C.c_double), ("rt_scheme", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        D, I, P = C.c_double, C.c_int, C.POINTER
        dp, ip, sp = P(C.c_double), P(C.c_int), P(OraScene)
        sig = {
            "ora_abi_version": (I, []),
            "ora_metric": (None, [sp, D, D, dp, dp]),
            "ora_dmetric": (None, [sp, D, D, dp]),
            "ora_connection": (None, [sp, D, D, dp]),
            "ora_step_size": (D, [sp, dp, dp]),
            "ora_rk4_step": (None, [sp, dp, dp, D]),
            "ora_verlet_step": (None, [sp, dp, dp, dp, D, I]),
            "ora_horizon": (D, [sp]),
            "ora_vec_bl_to_ks": (None, [sp, D, dp, dp]),
            "ora_pos_bl_to_ks": (None, [sp, dp, dp]),
            "ora_camera": (None, [sp, D, D, D, dp, dp]),
            "ora_constants": (None, [sp, dp, dp, dp]),
            "ora_r_isco": (D, [D]),
            "ora_newton_x2": (D, [D, D, D, ip]),
            "ora_grid_bilinear": (I, [sp, I, D, D, dp]),
            "ora_plasma": (I, [sp, dp, dp]),
            "ora_emissivity": (None, [D, D, D, D, D, I, dp]),
            "ora_rt_update": (None, [dp, dp, D, D, D, D]),
            "ora_trace_ray": (I, [sp, D, D, D, dp, I, dp, dp, ip, dp, I]),
            "ora_geodesic": (I, [sp, D, D, I, dp, dp, ip]),
            "ora_render": (I, [sp, dp, I, D, I, I, dp, ip, ip, I]),
            "ora_disk_ray": (I, [sp, D, D, D, D, D, I, dp]),
            "ora_disk_render": (I, [sp, D, D, D, I, dp, dp, ip, ip, ip, I]),
            "ora_disk_crossings": (I, [sp, D, D, I, dp, dp, dp, ip, ip]),
            "ora_length_unit_cm": (D, [D]),
            "ora_num_threads": (I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def scene(**kw) -> OraScene:
    """Scene with the defaults of the analytic workload (a=0.9, i=60 deg, r_cam=1000,
    64x64 over +-20 M, eps=0.05, M=4e6 Msun, D=7.88 kpc); keyword overrides."""
    s = OraScene()
    d = dict(m=1.0, a=0.9, coords=0, step_rule=0, r_cam=1000.0, incl_deg=60.0, nx=64, ny=64,
             amin=-20.0, amax=20.0, bmin=-20.0, bmax=20.0, eps=0.05, r_stop_factor=1.01,
             r_esc=1000.0, tau_cut=float("inf"), max_steps=100000, k2_exact=0,
             mass_msun=4.0e6, dist_pc=7.88e3, plasma_kind=KIND_ANALYTIC, slow_light=0,
             n0=1.0e6, n_pow=-1.5, the0=10.0, the_pow=-1.0, B0=20.0, B_pow=-1.0,
             ball_R=0.0, ball_j=0.0, ball_alpha=0.0, grid=None, n1=0, n2=0, n_snap=0, snap=0,
             x1_min=0.0, x1_max=0.0, h_mks=1.0, t0=0.0, dt_snap=1.0,
             mass_unit_g=0.0, r_high=1.0, r_low=1.0, gamma_ad=4.0 / 3.0, integrator=RK4, theta_e_min=0.0, rt_scheme=0)
    d.update(kw)
    keep = d.pop("_grid_ref", None)
    for k, v in d.items():
        setattr(s, k, v)
    s._keep = keep
    return s


def attach_grid(s: OraScene, grid: np.ndarray, x1_min: float, x1_max: float, h_mks: float) -> OraScene:
    """Point the scene at a float32 grid [n_snap][8][n2][n1] (kept alive on the scene)."""
    g = np.ascontiguousarray(grid, dtype=np.float32)
    s._keep = g
    s.grid = g.ctypes.data
    s.n_snap, _, s.n2, s.n1 = g.shape
    s.x1_min, s.x1_max, s.h_mks = x1_min, x1_max, h_mks
    s.plasma_kind = KIND_GRID
    return s


def metric(s, r, th):
    g = np.zeros(16); gi = np.zeros(16)
    lib().ora_metric(C.byref(s), r, th, _dp(g), _dp(gi))
    return g.reshape(4, 4), gi.reshape(4, 4)


def dmetric(s, r, th):
    dg = np.zeros(64)
    lib().ora_dmetric(C.byref(s), r, th, _dp(dg))
    return dg.reshape(4, 4, 4)


def connection(s, r, th):
    G = np.zeros(64)
    lib().ora_connection(C.byref(s), r, th, _dp(G))
    return G.reshape(4, 4, 4)


def camera(s, alpha, beta, t_cam=0.0):
    x = np.zeros(4); k = np.zeros(4)
    lib().ora_camera(C.byref(s), alpha, beta, t_cam, _dp(x), _dp(k))
    return x, k


def constants(s, x, k):
    """(E, L, Q, k.k) of the physical photon for the backward state (x, k)."""
    out = np.zeros(4)
    lib().ora_constants(C.byref(s), _dp(np.ascontiguousarray(x, float)), _dp(np.ascontiguousarray(k, float)), _dp(out))
    return out


def step_size(s, x, k):
    return lib().ora_step_size(C.byref(s), _dp(np.ascontiguousarray(x, float)), _dp(np.ascontiguousarray(k, float)))


def rk4_step(s, x, k, dl):
    x = np.array(x, float); k = np.array(k, float)
    lib().ora_rk4_step(C.byref(s), _dp(x), _dp(k), dl)
    return x, k


def verlet_step(s, x, k, f, dl, reeval=False):
    """One velocity-Verlet step (sec. 2.2.2); f is the carried derivative.  Returns (x, k, f)."""
    x = np.array(x, float); k = np.array(k, float); f = np.array(f, float)
    lib().ora_verlet_step(C.byref(s), _dp(x), _dp(k), _dp(f), dl, int(reeval))
    return x, k, f


def horizon(s):
    return lib().ora_horizon(C.byref(s))


def vec_bl_to_ks(s, r, vb):
    vb = np.ascontiguousarray(vb, float); vk = np.zeros(4)
    lib().ora_vec_bl_to_ks(C.byref(s), r, _dp(vb), _dp(vk))
    return vk


def pos_bl_to_ks(s, xb):
    xb = np.ascontiguousarray(xb, float); xk = np.zeros(4)
    lib().ora_pos_bl_to_ks(C.byref(s), _dp(xb), _dp(xk))
    return xk


def r_isco(a):
    return lib().ora_r_isco(a)


def newton_x2(theta, h, tol=1e-14):
    it = C.c_int(0)
    x = lib().ora_newton_x2(theta, h, tol, C.byref(it))
    return x, it.value


def grid_bilinear(s, snap, x1, x2):
    out = np.zeros(8)
    ok = lib().ora_grid_bilinear(C.byref(s), snap, x1, x2, _dp(out))
    return ok, out


def plasma(s, x):
    """(ok, n_e, Theta_e, B, u[4], b[4]) at KS position x."""
    out = np.zeros(11)
    ok = lib().ora_plasma(C.byref(s), _dp(np.ascontiguousarray(x, float)), _dp(out))
    return ok, out[0], out[1], out[2], out[3:7].copy(), out[7:11].copy()


def emissivity(nu, ne, thetae, B, sin_thb=1.0, k2_exact=0):
    """(j_nu, B_nu) of Eqs. 41-44 in CGS."""
    out = np.zeros(2)
    lib().ora_emissivity(nu, ne, thetae, B, sin_thb, k2_exact, _dp(out))
    return out[0], out[1]


def rt_update(I, tau, j, S, g, dl_cm):
    Ia = np.array([I], float); ta = np.array([tau], float)
    lib().ora_rt_update(_dp(Ia), _dp(ta), j, S, g, dl_cm)
    return Ia[0], ta[0]


def trace_ray(s, alpha, beta, freqs, t_cam=0.0, max_trace=0):
    """Trace one backward ray.  Returns dict(I, tau, steps, status, trace[n,12])."""
    nus = np.ascontiguousarray(freqs, float).ravel()
    nf = nus.size
    I = np.zeros(max(nf, 1)); tau = np.zeros(max(nf, 1)); n = C.c_int(0)
    tr = np.zeros((max(max_trace, 1), 12))
    st = lib().ora_trace_ray(C.byref(s), alpha, beta, t_cam, _dp(nus), nf, _dp(I), _dp(tau), C.byref(n),
                             _dp(tr) if max_trace > 0 else None, max_trace)
    return dict(I=I[:nf].copy(), tau=tau[:nf].copy(), steps=n.value, status=st,
                trace=tr[: min(n.value, max_trace)].copy() if max_trace > 0 else None)


def geodesic(s, alpha, beta, max_steps=100000):
    x = np.zeros(4); k = np.zeros(4); n = C.c_int(0)
    st = lib().ora_geodesic(C.byref(s), alpha, beta, max_steps, _dp(x), _dp(k), C.byref(n))
    return st, x, k, n.value


def render(s, freqs, t_cam=0.0, row0=0, nrows=0, nthreads=0):
    """Image [n_freq][rows][nx] in Jy/pixel, steps [rows][nx], status [rows][nx]."""
    nus = np.ascontiguousarray(freqs, float).ravel()
    nf = nus.size
    if nf > 64:
        raise ValueError("oracle render supports at most 64 frequencies")
    rows = s.ny if nrows <= 0 else nrows
    img = np.zeros((nf, rows, s.nx)); steps = np.zeros((rows, s.nx), np.int32)
    status = np.zeros((rows, s.nx), np.int32)
    lib().ora_render(C.byref(s), _dp(nus), nf, t_cam, row0, nrows, _dp(img), _ip(steps), _ip(status), nthreads)
    return img, steps, status


def disk_ray(s, alpha, beta, r_in=0.0, r_out=15.0, q=2.0, max_cross=10):
    """One ray against the thin disk of sec. 4.2.1 (r_in <= 0: the ISCO).  Returns dict(status,
    ratio = E_obs/E_em, I, order, r, theta, g, steps)."""
    out = np.zeros(7)
    st = lib().ora_disk_ray(C.byref(s), alpha, beta, r_in, r_out, q, max_cross, _dp(out))
    return dict(status=st, ratio=out[0], I=out[1], order=int(out[2]), r=out[3], theta=out[4], g=out[5],
                steps=int(out[6]))


def disk_crossings(s, alpha, beta, max_n=4):
    """Ordered equatorial crossings of one ray (the thin disk's geometry without the disk):
    dict(r, lam, t: arrays of the crossings found, fate: ESCAPED, CAPTURED, TRUNCATED, ERROR
    or CROSSINGS_MAX, steps)."""
    r = np.zeros(max(max_n, 1)); lam = np.zeros_like(r); t = np.zeros_like(r)
    fate = C.c_int(0); steps = C.c_int(0)
    n = lib().ora_disk_crossings(C.byref(s), alpha, beta, int(max_n), _dp(r), _dp(lam), _dp(t), C.byref(fate),
                                 C.byref(steps))
    return dict(r=r[:n].copy(), lam=lam[:n].copy(), t=t[:n].copy(), fate=fate.value, steps=steps.value)


def disk_render(s, r_in=0.0, r_out=15.0, q=2.0, max_cross=10, nthreads=0):
    """Thin-disk image: (ratio, I, order, status, steps), each [ny][nx]."""
    shape = (s.ny, s.nx)
    ratio = np.zeros(shape); inten = np.zeros(shape)
    order = np.zeros(shape, np.int32); status = np.zeros(shape, np.int32); steps = np.zeros(shape, np.int32)
    lib().ora_disk_render(C.byref(s), r_in, r_out, q, max_cross, _dp(ratio), _dp(inten), _ip(order), _ip(status),
                          _ip(steps), nthreads)
    return ratio, inten, order, status, steps


def line_profile(ratio, inten, order, x_min, x_max, n_bins, pix_area, profile_order=1):
    """Line spectrum of sec. 4.2.1: the sum of I * pixel area over pixels whose hit has
    crossing number profile_order (0: any order), in n_bins bins of E_obs/E_em over
    [x_min, x_max): bin floor((x - x_min) / dx), dx = (x_max - x_min) / n_bins."""
    sel = (order == profile_order) if profile_order > 0 else (order > 0)
    dx = (x_max - x_min) / n_bins
    hist = np.zeros(n_bins)
    for x, w in zip(ratio[sel].ravel(), inten[sel].ravel()):
        b = int(np.floor((x - x_min) / dx))
        if 0 <= b < n_bins:
            hist[b] += w * pix_area
    return hist


def length_unit_cm(mass_msun):
    return lib().ora_length_unit_cm(mass_msun)


def num_threads():
    return lib().ora_num_threads()
