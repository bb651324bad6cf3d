"""The host-side move-size tuner (geometric bisection of a common scale of
d and a on the acceptance of pilot runs), on a closed-form pilot and on the
oracle's ideal gas, whose acceptance is the in-cell probability
(1 - d / (2 w))^2 in 2D."""
import numpy as np

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs, tune


def test_bisection_on_a_monotone_pilot():
    calls = []

    def pilot(d, a):
        calls.append((d, a))
        return float(np.exp(-d))                      # acceptance falls as moves grow

    d, a, acc = tune.tune_scale(pilot, 0.2, 0.1, target=0.30, lo=0.25, hi=64.0, iters=30)
    assert abs(d - (-np.log(0.30))) < 1e-6 and abs(acc - 0.30) < 1e-6
    assert abs(a / d - 0.5) < 1e-12                   # the ratio d / a is kept
    assert len(calls) == 30 and all(abs(x[1] / x[0] - 0.5) < 1e-12 for x in calls)


def test_ideal_gas_acceptance_reaches_its_closed_form_size():
    L, w_min = 40.0, 1.0
    s = orc.OracleSystem(2, [L, L], inputs.regular_polygon(5, 1e-4), w_min=w_min)
    w = s.geometry()["w"][0]
    rng = np.random.default_rng(3)
    N = 3000
    pos0 = rng.uniform(0, L, (N, 2))
    th = rng.uniform(0, 2 * np.pi, N)
    ori0 = np.stack([np.cos(th), np.sin(th)], 1)

    def pilot(d, a):
        s.set_moves(d, a, 4, 5)
        p, o = pos0.copy(), ori0.copy()
        c = s.sweep(p, o, 0, 10)
        return c[0] / (c[0] + c[1] + c[2])

    target = 0.30
    d, a, acc = tune.tune_scale(pilot, 0.1, 0.1, target=target, lo=0.25, hi=16.0, iters=14)
    d_exact = 2 * w * (1 - np.sqrt(target))
    assert abs(d - d_exact) < 0.02 * d_exact, (d, d_exact)
    assert abs(acc - target) < 0.01 and a == d
