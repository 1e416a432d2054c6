"""Workload definitions and seeded synthetic inputs.

Shared by the tests (which feed the same inputs to the oracle and to the CUDA library) and
by the benchmark.  Holds parameters and input generation only -- none of the ray-tracing
or transfer arithmetic.
"""
from __future__ import annotations

import numpy as np

# Sgr A*-like units of the slow-light study (sec. 5): M = 4e6 Msun, D = 7.88 kpc.
MASS_MSUN = 4.0e6
DIST_PC = 7.88e3

# Analytic scene: n_e = 1e6 r^-1.5 cm^-3, Theta_e = 10 / r, B = 20 G / r.
ANALYTIC_PLASMA = dict(n0=1.0e6, n_pow=-1.5, the0=10.0, the_pow=-1.0, B0_gauss=20.0, B_pow=-1.0)

# Small analytic image: a = 0.9, i = 60 deg, r_cam = 1000 M, 64 x 64 over +-20 M, 230 GHz.
SMALL = dict(spin=0.9, incl_deg=60.0, r_cam=1000.0, nx=64, ny=64, alpha_min=-20.0, alpha_max=20.0,
             beta_min=-20.0, beta_max=20.0, eps=0.05, r_stop_factor=1.01, r_escape=1000.0,
             mass_msun=MASS_MSUN, distance_pc=DIST_PC)
SMALL_FREQS = [230e9]

# Eight log-spaced frequencies 1e10 .. 1e13 Hz and three spins, 512 x 512.
SPECTRAL_FREQS = [1e10 * 10 ** (3 * k / 7) for k in range(8)]
SPECTRAL_SPINS = [0.0, 0.5, 0.9375]
SPECTRAL = dict(SMALL, nx=512, ny=512)

# Headline image: 1024 x 1024, a = 0.9375, i = 60 deg, 230 GHz.
HEADLINE = dict(SMALL, spin=0.9375, nx=1024, ny=1024)

# Thin-disk line emitter (sec. 4.2.1): disk from the ISCO to 15 M, emission ~ r^-2, the
# paper's five spins; 1024^2 over +-16 M at i = 30 deg (the paper does not state i).
THIN_DISK = dict(SMALL, spin=0.99, incl_deg=30.0, nx=1024, ny=1024, alpha_min=-16.0, alpha_max=16.0,
                 beta_min=-16.0, beta_max=16.0)
THIN_DISK_GEOM = dict(r_out=15.0, q=2.0, max_cross=10)
THIN_DISK_SPINS = [-0.99, -0.5, 0.0, 0.5, 0.99]
HEADLINE_FREQS = [230e9]


def sample_pixels(nx: int, ny: int, n: int, seed: int) -> np.ndarray:
    """Seeded sample of n distinct pixel indices (row, col)."""
    rng = np.random.default_rng(seed)
    flat = rng.choice(nx * ny, size=min(n, nx * ny), replace=False)
    return np.stack([flat // nx, flat % nx], axis=1)


# ---------------------------------------------------------------------------------------
# Synthetic GRMHD-shaped snapshots (inputs of the grid workloads).
#
# A Fishbone & Moncrief (1976) torus around a Kerr hole (constant l = u^t u_phi, inner edge
# r_in, pressure maximum r_max), polytropic gas, a poloidal field loop following the
# density, a power-law atmosphere, and a mean-preserving lognormal noise field
# exp(sigma G - sigma^2/2) on rho and u, where G is a unit-variance Gaussian random field
# with squared-exponential correlation length ell (random Fourier features), sampled on the
# phi = 0 meridional plane.  Snapshot s of a time series samples G at points rotated about
# the spin axis by -Omega_K(varpi) t_s, so the noise is advected at the local Keplerian
# angular velocity.  Output: float32 [n_snap][8][n2][n1] HARM primitives on a cell-centred
# MKS grid (x1 = ln r, theta = pi x2 + (1-h)/2 sin 2 pi x2): rho, u, U1, U2, U3, B1, B2, B3.
# ---------------------------------------------------------------------------------------
TORUS = dict(spin=0.9375, r_in=6.0, r_max=12.0, n1=256, n2=256, h_mks=0.3, r_out=50.0, gamma_ad=4.0 / 3.0,
             kappa=1e-3, beta_min=100.0, sigma=0.5, ell=2.0, n_modes=512, seed=0x1801104520000003)
SLOW = dict(TORUS, n_snap=100, dt_snap=10.0, seed=0x1801104520000004)
# Disk-dominated model of sec. 5.2: mass unit 5.03e-15 Msun (in grams), R_high = R_low = 1.
MSUN_G = 1.98841e33
DISK_MODEL = dict(mass_unit_g=5.03e-15 * MSUN_G, r_high=1.0, r_low=1.0)


def _kerr_bl(a, r, th):
    s2 = np.sin(th) ** 2
    Sig = r * r + a * a * np.cos(th) ** 2
    Del = r * r - 2 * r + a * a
    A = (r * r + a * a) ** 2 - Del * a * a * s2
    return Sig, Del, A, s2


def _fm_lnh(a, l, r, th, r_in):
    """ln h of the FM torus (h = specific enthalpy), zero at (r_in, pi/2)."""
    def raw(r, th):
        Sig, Del, A, s2 = _kerr_bl(a, r, th)
        E = Sig * Sig * Del / (A * A * s2)
        q = np.sqrt(1 + 4 * l * l * E)
        return 0.5 * np.log((1 + q) / (Sig * Del / A)) - 0.5 * q - 2 * a * r * l / A
    return raw(r, th) - raw(np.asarray(r_in, float), np.asarray(np.pi / 2))


def fm_angular_momentum(a, r_max):
    """l = u^t u_phi of the prograde circular equatorial geodesic at r_max."""
    sr = np.sqrt(r_max)
    return (r_max ** 1.5 + a) * (r_max ** 2 - 2 * a * sr + a * a) / (r_max ** 1.5 * (r_max ** 1.5 - 3 * sr + 2 * a))


def mks_grid(n1, n2, a, h, r_out):
    r_h = 1 + np.sqrt(1 - a * a)
    x1_min, x1_max = np.log(1.01 * r_h), np.log(r_out)
    x1 = x1_min + (np.arange(n1) + 0.5) * (x1_max - x1_min) / n1
    x2 = (np.arange(n2) + 0.5) / n2
    X1, X2 = np.meshgrid(x1, x2)  # [n2][n1]
    r = np.exp(X1)
    th = np.pi * X2 + 0.5 * (1 - h) * np.sin(2 * np.pi * X2)
    return dict(x1_min=x1_min, x1_max=x1_max, r=r, th=th, x2=X2)


def _noise(rng, n_modes, ell):
    k = rng.normal(size=(n_modes, 3)) / ell
    ph = rng.uniform(0, 2 * np.pi, n_modes)
    return k.astype(np.float64), ph


def _sample_noise(k, ph, X, device=None):
    """G at points X [..., 3]: sqrt(2/N) sum cos(k.x + phi).  With a torch `device` the sum
    runs there in float64 (same formula; rounding differs in the last bits)."""
    shp = X.shape[:-1]
    if device is not None:
        import torch

        kt = torch.as_tensor(k, dtype=torch.float64, device=device)
        pt = torch.as_tensor(ph, dtype=torch.float64, device=device)
        P = torch.as_tensor(X.reshape(-1, 3), dtype=torch.float64, device=device)
        g = torch.cos(P @ kt.T + pt).sum(1) * np.sqrt(2.0 / k.shape[0])
        return g.cpu().numpy().reshape(shp)
    P = X.reshape(-1, 3)
    out = np.empty(P.shape[0])
    for i in range(0, P.shape[0], 16384):
        arg = P[i:i + 16384] @ k.T + ph
        out[i:i + 16384] = np.cos(arg).sum(1)
    return (np.sqrt(2.0 / k.shape[0]) * out).reshape(shp)


def torus_snapshots(n_snap=1, dt_snap=10.0, device=None, **over):
    """Seeded synthetic snapshot series.  Returns (fields float32 [n_snap][8][n2][n1], meta).
    device: a torch device for the noise sums (long series; default numpy)."""
    c = dict(TORUS)
    c.update(over)
    a, h, gam = c["spin"], c["h_mks"], c["gamma_ad"]
    G = mks_grid(c["n1"], c["n2"], a, h, c["r_out"])
    r, th, x2 = G["r"], G["th"], G["x2"]
    l = fm_angular_momentum(a, c["r_max"])
    lnh = _fm_lnh(a, l, r, th, c["r_in"])
    inside = (lnh > 0) & (r >= c["r_in"])
    hm1 = np.where(inside, np.expm1(np.where(inside, lnh, 0.0)), 0.0)
    rho_t = np.where(inside, (hm1 * (gam - 1) / (c["kappa"] * gam)) ** (1 / (gam - 1)), 0.0)
    rho_t /= rho_t.max()
    # polytrope: P / rho = (h - 1)(gamma - 1)/gamma, so u / rho = (h - 1) / gamma whatever the
    # density normalisation
    u_t = rho_t * hm1 / gam
    # FM velocity (BL: u^r = u^theta = 0), then the KS normal-observer primitives
    Sig, Del, A, s2 = _kerr_bl(a, r, th)
    E = Sig * Sig * Del / (A * A * s2)
    U2 = 0.5 * (-1 + np.sqrt(1 + 4 * l * l * E))
    U = np.sqrt(U2)
    alpha_bl = np.sqrt(Sig * Del / A)
    omega = 2 * a * r / A
    gpp = A * s2 / Sig
    ut = np.sqrt(1 + U2) / alpha_bl
    uphi = ut * omega + U / np.sqrt(gpp)
    z = 2 * r / Sig
    Ur_ks = ut * z / (1 + z)
    U1 = np.where(inside, Ur_ks / r, 0.0)
    U3 = np.where(inside, uphi, 0.0)
    # poloidal loop: A_phi ~ max(rho/rho_max - 0.2, 0); B^i = eps^{ijk} d_j A_k / sqrt(-g) (MKS)
    Aphi = np.maximum(rho_t - 0.2, 0.0)
    dx1 = (G["x1_max"] - G["x1_min"]) / c["n1"]
    dx2 = 1.0 / c["n2"]
    dA_dx2, dA_dx1 = np.gradient(Aphi, dx2, dx1)
    dth_dx2 = np.pi * (1 + (1 - h) * np.cos(2 * np.pi * x2))
    gdet = Sig * np.sqrt(s2) * r * dth_dx2
    B1 = -dA_dx2 / gdet
    B2 = dA_dx1 / gdet
    B3 = np.zeros_like(B1)
    # normalise to max P_gas / max P_mag = beta_min (P_mag ~ g_ij B^i B^j / 2, KS radial part)
    bsq = (1 + z) * (r * B1) ** 2 + Sig * (dth_dx2 * B2) ** 2
    pg = (gam - 1) * u_t
    if bsq.max() > 0:
        norm = np.sqrt(pg.max() / (0.5 * bsq.max()) / c["beta_min"])
        B1 *= norm
        B2 *= norm
    # atmosphere
    rho_fl = 1e-4 * r ** -1.5
    u_fl = 1e-6 * r ** -2.5
    rng = np.random.default_rng(c["seed"])
    k, ph = _noise(rng, c["n_modes"], c["ell"])
    varpi = r * np.sqrt(s2)
    Om_k = 1.0 / (varpi ** 1.5 + a)
    out = np.empty((n_snap, 8, c["n2"], c["n1"]), np.float32)
    for s in range(n_snap):
        ang = -Om_k * dt_snap * s
        X = np.stack([varpi * np.cos(ang), varpi * np.sin(ang), r * np.cos(th)], -1)
        Gn = _sample_noise(k, ph, X, device)
        ln = np.exp(c["sigma"] * Gn - 0.5 * c["sigma"] ** 2)
        rho = np.maximum(rho_t * ln, rho_fl)
        u = np.maximum(u_t * ln, u_fl)
        out[s] = np.stack([rho, u, U1, np.zeros_like(U1), U3, B1, B2, B3]).astype(np.float32)
    meta = dict(x1_min=G["x1_min"], x1_max=G["x1_max"], h_mks=h, n1=c["n1"], n2=c["n2"], n_snap=n_snap,
                dt_snap=dt_snap, gamma_ad=gam, spin=a, l=l)
    return out, meta


def grid_plasma(meta: dict, model: dict, slow: int = 0, t0: float = 0.0) -> dict:
    """raptor_plasma_desc fields of a grid snapshot series made by torus_snapshots."""
    return dict(slow_light=slow, x1_min=meta["x1_min"], x1_max=meta["x1_max"], h_mks=meta["h_mks"], t0=t0,
                dt_snap=meta["dt_snap"], mass_unit_g=model["mass_unit_g"], r_high=model["r_high"],
                r_low=model["r_low"], gamma_ad=meta["gamma_ad"])
