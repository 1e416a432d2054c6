"""Shared test helpers (no ray-tracing arithmetic of either implementation)."""
import math

import numpy as np


def bardeen_critical_curve(a, incl_deg, n=2000):
    """Closed-form critical curve on the observer's sky (Bardeen 1973): points (alpha, beta)
    for photon-orbit radii between the prograde and retrograde circular photon orbits."""
    if abs(a) < 1e-9:
        t = np.linspace(0, 2 * np.pi, n)
        b = 3 * math.sqrt(3)
        return np.stack([b * np.cos(t), b * np.sin(t)], 1)
    rp = 2 * (1 + math.cos(2 / 3 * math.acos(-abs(a))))
    rm = 2 * (1 + math.cos(2 / 3 * math.acos(abs(a))))
    r = np.linspace(rp, rm, n)
    xi = -(r**3 - 3 * r**2 + a * a * r + a * a) / (a * (r - 1))
    eta = r**3 * (4 * a * a - r * (r - 3) ** 2) / (a * a * (r - 1) ** 2)
    ci, si = math.cos(math.radians(incl_deg)), math.sin(math.radians(incl_deg))
    b2 = eta + a * a * ci * ci - xi * xi * ci * ci / (si * si)
    m = b2 >= 0
    al = -xi[m] / si
    be = np.sqrt(b2[m])
    return np.concatenate([np.stack([al, be], 1), np.stack([al[::-1], -be[::-1]], 1)])


def ring_mask(alpha, beta, a, incl_deg, width):
    """True for pixel centres within `width` M of the critical curve."""
    cc = bardeen_critical_curve(a, incl_deg)
    A, B = np.meshgrid(alpha, beta)
    P = np.stack([A.ravel(), B.ravel()], 1)
    d = np.full(P.shape[0], np.inf)
    for i in range(0, cc.shape[0], 256):
        c = cc[i:i + 256]
        d = np.minimum(d, np.sqrt(((P[:, None, :] - c[None, :, :]) ** 2).sum(-1)).min(1))
    return (d < width).reshape(A.shape)


def near_ring(alpha, beta, a, incl_deg, width):
    """True for the points (alpha[n], beta[n]) within `width` M of the critical curve."""
    cc = bardeen_critical_curve(a, incl_deg)
    P = np.stack([np.asarray(alpha, float), np.asarray(beta, float)], 1)
    d = np.sqrt(((P[:, None, :] - cc[None, :, :]) ** 2).sum(-1)).min(1)
    return d < width


def rel_err(gpu, ref, floor_frac=1e-12):
    """|gpu - ref| / max(|ref|, floor_frac * max|ref|) element-wise."""
    ref = np.asarray(ref)
    den = np.maximum(np.abs(ref), floor_frac * np.abs(ref).max())
    return np.abs(np.asarray(gpu) - ref) / den


def oracle_kwargs(cam: dict, plasma: dict | None = None) -> dict:
    """Translate a camera/plasma parameter dict into the oracle's scene keywords."""
    from paper_1801_10452_b300.scenes import ANALYTIC_PLASMA

    pl = dict(ANALYTIC_PLASMA if plasma is None else plasma)
    out = dict(a=cam["spin"], incl_deg=cam["incl_deg"], r_cam=cam["r_cam"], nx=cam["nx"], ny=cam["ny"],
               amin=cam["alpha_min"], amax=cam["alpha_max"], bmin=cam["beta_min"], bmax=cam["beta_max"],
               eps=cam["eps"], r_stop_factor=cam["r_stop_factor"], r_esc=cam["r_escape"],
               mass_msun=cam["mass_msun"], dist_pc=cam["distance_pc"],
               n0=pl["n0"], n_pow=pl["n_pow"], the0=pl["the0"], the_pow=pl["the_pow"], B0=pl["B0_gauss"],
               B_pow=pl["B_pow"])
    for k in ("max_steps", "tau_cut"):
        if k in cam:
            out[k] = cam[k]
    return out


def grid_oracle_scene(ora, cam, fields, meta, model, slow=0, t0=0.0, snap=0):
    """Oracle scene for a grid workload (same arrays the library receives)."""
    kw = oracle_kwargs(cam)
    s = ora.scene(**kw)
    ora.attach_grid(s, fields, meta["x1_min"], meta["x1_max"], meta["h_mks"])
    s.mass_unit_g = model["mass_unit_g"]
    s.r_high = model["r_high"]
    s.r_low = model["r_low"]
    s.gamma_ad = meta["gamma_ad"]
    s.t0 = t0
    s.dt_snap = meta["dt_snap"]
    s.slow_light = slow
    s.snap = snap
    return s


def grid_plasma_kwargs(meta, model, slow=0, t0=0.0):
    from paper_1801_10452_b300 import scenes

    return scenes.grid_plasma(meta, model, slow, t0)
