"""The histogram extrapolation of the pressure estimator, pinned on
synthetic histograms whose limit at x = 0 is known in closed form."""
import math

import numpy as np
import pytest

from paper_1509_04692_gb300 import pressure


@pytest.mark.parametrize("h0,k", [(2000.0, 12.0), (500.0, -4.0), (8000.0, 30.0)])
def test_extrapolation_recovers_exponential_limit(h0, k):
    # expected counts of n configurations with h(x) = h0 exp(-k x), integrated per bin
    n, x_max, nb = 100, 0.05, 25
    edges = np.linspace(0.0, x_max, nb + 1)
    if k == 0:
        counts = h0 * n * np.diff(edges)
    else:
        counts = h0 * n * (np.exp(-k * edges[:-1]) - np.exp(-k * edges[1:])) / k
    got, err = pressure.extrapolate_h0(counts, n, x_max, deg=2)
    assert abs(got - h0) < 1e-3 * h0
    assert err > 0


def test_pressure_of_contact_value():
    # 2D: dn/dx at 0 = N pi rho sigma^2 g(sigma), so beta P / rho = 1 + (pi/2) rho sigma^2 g(sigma)
    N, L, g = 1000, 40.0, 1.3
    rho = N / L ** 2
    h0 = N * math.pi * rho * g
    counts = np.full(20, h0 * 50 * 0.05 / 20)              # flat histogram, 50 configurations
    out = pressure.pressure(counts, 50, 0.05, N, L * L, 2, deg=1)
    assert abs(out["beta_P_over_rho"] - (1 + 0.5 * math.pi * rho * g)) < 1e-9
    assert abs(out["P_star"] - out["beta_P_over_rho"] * rho) < 1e-12
