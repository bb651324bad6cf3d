"""Host-side move-size tuning (Sec. 2.1: moves sized for a target acceptance,
then fixed for production).

The translation half-width d and rotation parameter a are scaled together
(their ratio fixed) by bisection on the acceptance ratio of short pilot runs.
`pilot(d, a)` runs a pilot from a fixed starting state and returns the
acceptance ratio; any implementation of the sweep can serve as the pilot
because the acceptance is a property of the chain, not of the code.
"""
from __future__ import annotations


def tune_scale(pilot, d0: float, a0: float, target: float = 0.30, lo: float = 0.25,
               hi: float = 8.0, iters: int = 14):
    """Return (d, a, acceptance) with acceptance(d, a) closest to `target`."""
    best = None
    for _ in range(iters):
        mid = (lo * hi) ** 0.5
        acc = pilot(d0 * mid, a0 * mid)
        if best is None or abs(acc - target) < abs(best[2] - target):
            best = (d0 * mid, a0 * mid, acc)
        if acc > target:
            lo = mid            # moves too small: acceptance too high
        else:
            hi = mid
    return best
