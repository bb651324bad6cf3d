"""CPU pin of the O(N^2) pair count the GPU overlap counts are compared with:
on configurations with pairs planted across the periodic boundaries it
agrees with the brute-force polygon predicate (edge crossings and
point-in-polygon, a different minimum-image formula)."""
import numpy as np

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests import bruteforce as bf
from tests.paircount import oracle_pair_count, plant_wrap_pairs


def test_pair_count_matches_bruteforce_across_the_wrap():
    s = inputs.pentagon_system(1500, 0.45, seed=5)
    ref = orc.OracleSystem(2, s.L, s.verts)
    assert oracle_pair_count(ref, s.pos, s.orient) == 0
    for seed in range(3):
        p = plant_wrap_pairs(s.pos, s.L, seed=seed)
        got = oracle_pair_count(ref, p, s.orient)
        pairs = bf.pairwise_overlaps_2d(s.verts, np.asarray(s.L), p, s.orient)
        assert got == len(pairs)
        # the pairs straddling the x wrap, the y wrap and the corner
        assert {(0, 1), (2, 3), (4, 5)} <= set(pairs)
