"""Test-side statement of the pressure extrapolation (numpy least squares),
used by the oracle's pressure pins and compared with the library's
hpmc_pressure.

Pressure of hard particles from the scale-distribution histogram (Sec. 4
of Anderson, Irrgang & Glotzer; the volume perturbation that extends it to
particles with shape).

Compressing every position by the factor (1 - x), shapes unchanged, makes a
pair touch at some x* (disks / spheres: x* = 1 - sigma / r).  With h(x) the number of pairs per unit x
(per configuration) whose x* lies just above x, the volume-perturbation
argument gives beta P / rho = 1 + h(0) / (dim N): the probability that a
compression by x creates an overlap is h(0) x for small x, and the volume
changes by dim x V.  h(0) is extrapolated from the bins by a weighted
polynomial fit of log h.
"""
from __future__ import annotations

import math

import numpy as np


def extrapolate_h0(hist, n_samples: int, x_max: float, deg: int = 3):
    """h(0) and its standard error from a histogram of n_samples
    configurations over [0, x_max): weighted least squares of log h on the
    bin centres (Poisson weights), evaluated at x = 0."""
    hist = np.asarray(hist, dtype=np.float64)
    nb = hist.size
    dx = x_max / nb
    x = (np.arange(nb) + 0.5) * dx
    ok = hist > 0
    if ok.sum() <= deg + 1:
        raise ValueError("too few populated bins to extrapolate")
    y = np.log(hist[ok] / (n_samples * dx))
    w = np.sqrt(hist[ok])                      # 1 / sigma of log counts
    A = np.vander(x[ok], deg + 1, increasing=True)
    Aw = A * w[:, None]
    coef, *_ = np.linalg.lstsq(Aw, y * w, rcond=None)
    cov = np.linalg.inv(Aw.T @ Aw)
    h0 = math.exp(coef[0])
    return h0, h0 * math.sqrt(cov[0, 0])


def pressure(hist, n_samples: int, x_max: float, N: int, volume: float, dim: int, sigma: float = 1.0,
             deg: int = 3) -> dict:
    """Reduced pressure from an accumulated histogram: beta P / rho, and P*
    as the paper reports it for disks / spheres of diameter sigma (2D:
    beta P sigma^2; 3D: beta P v0 with v0 the sphere volume)."""
    h0, dh0 = extrapolate_h0(hist, n_samples, x_max, deg)
    bpr = 1.0 + h0 / (dim * N)
    rho = N / volume
    ref = sigma ** 2 if dim == 2 else math.pi / 6.0 * sigma ** 3
    return {"beta_P_over_rho": bpr, "beta_P_over_rho_err": dh0 / (dim * N),
            "P_star": bpr * rho * ref, "P_star_err": dh0 / (dim * N) * rho * ref, "h0": h0}
