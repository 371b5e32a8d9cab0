"""Host-side pieces of bench.py: the graphlet-incidence figure and the
multi-core oracle baseline (no GPU)."""
from math import comb

import numpy as np

import bench
import oracle
import synth


def test_incidences_from_numerator_sums_equal_the_per_edge_definition():
    rp, col = synth.chung_lu(3000, 20000, 2.1, 300.0, seed=4)
    pairs = synth.upper_pairs(rp, col)
    lc = oracle.local_counts(rp, col, pairs)
    direct = 0
    for t, a, b, k, q in zip(*(lc[x].tolist() for x in ("t", "a", "b", "k", "q"))):
        direct += (t + a + b + k + comb(t, 2) + t * (a + b) + q + comb(a, 2) + comb(b, 2)
                   + a * b)
    s, _ = oracle.numerators(lc)
    assert bench.incidences_from_numerators(s) == direct


def test_parallel_oracle_baseline_counts_a_bounded_sample_of_every_part():
    rp, col = synth.er(3000, 60000, seed=2)
    parts = [("exact_3node", 1.0, bench.THREE), ("0.01", 0.01, bench.CONN)]
    rates, cores = bench.oracle_part_rates(rp, col, parts, 0.4, seed=3, workers=2)
    assert cores == 2
    assert 0 < rates["0.01"][0] <= len(oracle.sample(rp, col, 0.01, 3))
    assert 0 < rates["exact_3node"][0] <= len(col) // 2
    assert all(w > 0 for _, w in rates.values())
    v, cores, sample, wall = bench.oracle_step_rate(rp, col, parts, 0.4, seed=3)
    assert np.isfinite(v) and v > 0 and "exact_3node" in sample
