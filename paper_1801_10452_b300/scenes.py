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
HEADLINE_FREQS = [230e9]


def sample_pixels(nx: int, ny: int, n: int, seed: int) -> np.ndarray:
    """Seeded sample of n distinct pixel indices (row, col)."""
    rng = np.random.default_rng(seed)
    flat = rng.choice(nx * ny, size=min(n, nx * ny), replace=False)
    return np.stack([flat // nx, flat % nx], axis=1)
