"""Pressure of hard particles from the scale-distribution histogram (Sec. 4
of Anderson, Irrgang & Glotzer): marshalling for the library's
hpmc_pressure, which extrapolates h(0) (weighted least squares of log h on
the bin centres) and returns beta P / rho = 1 + h(0) / (dim N).  The default
degree is cubic: a quadratic underestimates the solid's curvature near
contact (hard spheres at volume fraction 0.60 read 0.01 low with it).
"""
from __future__ import annotations

from . import hpmc


def extrapolate_h0(hist, n_samples: int, x_max: float, deg: int = 3):
    """h(0) and its standard error from a histogram of n_samples
    configurations over [0, x_max)."""
    out = hpmc.pressure(hist, n_samples, x_max, 1, 1.0, 2, deg=deg)
    return out["h0"], out["h0_err"]


def pressure(hist, n_samples: int, x_max: float, N: int, volume: float, dim: int, sigma: float = 1.0,
             deg: int = 3) -> dict:
    """Reduced pressure from an accumulated histogram: beta P / rho, and P*
    as the paper reports it for disks / spheres of diameter sigma (2D:
    beta P sigma^2; 3D: beta P v0 with v0 the sphere volume)."""
    return hpmc.pressure(hist, n_samples, x_max, N, volume, dim, sigma=sigma, deg=deg)
