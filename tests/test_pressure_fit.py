"""The library's pressure extrapolation (hpmc_pressure, Sec. 4), called
through the C ABI on the host: pinned on synthetic histograms whose limit at
x = 0 is known in closed form, on the contact-value formula, and against the
test-side numpy least-squares statement on random histograms."""
import math

import numpy as np
import pytest

from tests import pressure_ref

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")


@pytest.mark.parametrize("h0,k", [(2000.0, 12.0), (500.0, -4.0), (8000.0, 30.0)])
def test_extrapolation_recovers_exponential_limit(h0, k):
    # expected counts of n configurations with h(x) = h0 exp(-k x), integrated
    # per bin (rounded to whole counts; n large so that rounding is tiny).
    # A bin's mean of h is h at its centre times sinh(k dx / 2) / (k dx / 2)
    # for every bin, so log h of the bins is exactly linear and the fit's
    # value at 0 is h0 times that factor.
    n, x_max, nb = 100000, 0.05, 25
    dx = x_max / nb
    edges = np.linspace(0.0, x_max, nb + 1)
    counts = np.rint(h0 * n * (np.exp(-k * edges[:-1]) - np.exp(-k * edges[1:])) / k)
    want = h0 * math.sinh(k * dx / 2) / (k * dx / 2)
    for deg in (1, 2, 3):
        out = hpmc.pressure(counts, n, x_max, 1000, 100.0, 2, deg=deg)
        assert abs(out["h0"] - want) < 2e-5 * want, (deg, out["h0"], want)
        assert out["h0_err"] > 0


def test_pressure_of_contact_value():
    # 2D: dn/dx at 0 = N pi rho sigma^2 g(sigma), so beta P / rho = 1 + (pi/2) rho sigma^2 g(sigma)
    N, L, n = 1000, 40.0, 64
    rho = N / L ** 2
    counts = np.full(20, 400.0)                            # flat histogram: h = 400 / (n dx)
    h0 = 400.0 / (n * 0.05 / 20)
    g = h0 / (N * math.pi * rho)                           # the contact value it stands for
    out = hpmc.pressure(counts, n, 0.05, N, L * L, 2, deg=1)
    assert abs(out["beta_P_over_rho"] - (1 + 0.5 * math.pi * rho * g)) < 1e-12
    assert abs(out["P_star"] - out["beta_P_over_rho"] * rho) < 1e-12
    # 3D: P* = beta P v0 with v0 = pi sigma^3 / 6
    out3 = hpmc.pressure(counts, n, 0.05, N, 1000.0, 3, sigma=1.3, deg=1)
    assert abs(out3["P_star"] - out3["beta_P_over_rho"] * (N / 1000.0) * math.pi / 6 * 1.3 ** 3) < 1e-12


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 5])
def test_library_fit_equals_the_numpy_statement(deg):
    rng = np.random.default_rng(deg)
    for _ in range(5):
        nb = int(rng.integers(10, 40))
        lam = 300 * np.exp(-rng.uniform(-20, 20) * np.linspace(0, 0.05, nb))
        counts = rng.poisson(lam).astype(np.float64)
        counts[rng.integers(0, nb)] = 0.0                   # an empty bin is left out
        n, N, V = int(rng.integers(1, 500)), int(rng.integers(100, 10 ** 6)), float(rng.uniform(10, 1e6))
        for dim in (2, 3):
            got = hpmc.pressure(counts, n, 0.05, N, V, dim, sigma=1.0, deg=deg)
            want = pressure_ref.pressure(counts, n, 0.05, N, V, dim, deg=deg)
            for key in ("beta_P_over_rho", "P_star", "h0"):
                assert abs(got[key] - want[key]) <= 1e-9 * abs(want[key]), (key, got[key], want[key])
            assert abs(got["beta_P_over_rho_err"] - want["beta_P_over_rho_err"]) <= \
                1e-6 * want["beta_P_over_rho_err"]


def test_invalid_arguments_are_refused():
    c = np.full(10, 100.0)
    for args in ((c, 0, 0.05, 10, 1.0, 2), (c, 10, 0.0, 10, 1.0, 2), (c, 10, 0.05, 0, 1.0, 2),
                 (c, 10, 0.05, 10, -1.0, 2), (c, 10, 0.05, 10, 1.0, 4)):
        with pytest.raises(hpmc.HPMCError):
            hpmc.pressure(*args)
    with pytest.raises(hpmc.HPMCError):                      # too few populated bins for the degree
        hpmc.pressure(np.array([5.0, 0, 0, 7.0]), 10, 0.05, 10, 1.0, 2, deg=2)
