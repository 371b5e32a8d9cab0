"""The sample-size formula of Sec. 6.2, K = (z sqrt(Var) / margin)^2, read with
the per-edge standard deviation of a pilot sample, a margin of rel_err |X|
and the finite-population correction.

Pins: (1) a target margin equal to the pilot's own half-width z sqrt(V)
asks for the pilot's own size (the variance formula inverted); (2) samples
of the size the formula asks for meet the target: about 95% of estimates
fall within rel_err of the exact count. The library's FP64 evaluation
equals the oracle's exact rational one, except by one where the exact value
lies within 1e-9 (relative) of an integer (the FP64 ceiling may land on
either side)."""
import math
from fractions import Fraction

import numpy as np

import oracle
import synth


def test_margin_equal_to_the_pilot_half_width_gives_the_pilot_size():
    rp, col = synth.chung_lu(3000, 20000, 2.1, 300.0, seed=5)
    m = len(col) // 2
    pairs = oracle.sample(rp, col, 0.05, 4)
    k = len(pairs)
    s, s2 = oracle.numerators(oracle.local_counts(rp, col, pairs))
    est = oracle.estimate(s, s2, m, k)
    for g in oracle.GRAPHLETS:
        if est[g]["X"] == 0 or est[g]["V"] == 0:
            continue
        rel = 1.96 * math.sqrt(est[g]["V"]) / abs(est[g]["X"])
        got = oracle.sample_size(s, s2, m, k, rel)[g]
        assert abs(got - k) <= 1, (g, got, k)


def test_samples_of_the_requested_size_meet_the_target():
    rp, col = synth.er(600, 9000, seed=8)
    m = len(col) // 2
    exact = oracle.exact_counts(rp, col)
    pilot = oracle.sample(rp, col, 0.02, 1)
    s, s2 = oracle.numerators(oracle.local_counts(rp, col, pilot))
    need = oracle.sample_size(s, s2, m, len(pilot), 0.10)
    up = synth.upper_pairs(rp, col)
    lc_all = oracle.local_counts(rp, col, up)
    rng = np.random.default_rng(3)
    for g in (3, 4, 9, 12):
        K = need[g]
        assert 1 < K < m
        inside = 0
        trials = 400
        for _ in range(trials):
            idx = rng.choice(m, size=K, replace=False)
            sub = {x: v[idx] for x, v in lc_all.items()}
            ss, ss2 = oracle.numerators(sub)
            x = oracle.estimate(ss, ss2, m, K)[g]["X"]
            inside += abs(x - exact[g]) <= 0.10 * exact[g]
        # the pilot's spread only estimates the population's: 95% +- 5 points
        assert 0.88 * trials <= inside <= trials, (g, K, inside)


def test_library_sample_size_equals_the_oracle():
    import paper_1701_01772_gb300 as gs
    gs.build()
    rp, col = synth.chung_lu(5000, 40000, 2.1, 400.0, seed=2)
    m = len(col) // 2
    for frac, seed, rel in ((0.01, 1, 0.05), (0.05, 2, 0.01), (0.2, 3, 0.2), (0.5, 4, 0.001)):
        pairs = oracle.sample(rp, col, frac, seed)
        s, s2 = oracle.numerators(oracle.local_counts(rp, col, pairs))
        want = oracle.sample_size(s, s2, m, len(pairs), rel)
        got = gs.gs_sample_size(gs.sums_from_ints(len(pairs), m, gs.GS_CONNECTED, s, s2), rel)
        for g in oracle.GRAPHLETS:
            if got[g] == want[g]:
                continue
            # the exact value lies within 1e-9 of the integer the ceilings split at
            d = oracle.DENOM[g]
            k = len(pairs)
            S2 = Fraction(k * s2[g] - s[g] * s[g], k * (k - 1) * d * d)
            X = Fraction(m * s[g], k * d)
            h = Fraction(rel) * abs(X)
            n0 = Fraction(1.96) ** 2 * m * m * S2 / (h * h)
            exact = n0 / (1 + n0 / m)
            assert abs(got[g] - want[g]) == 1, (g, got[g], want[g])
            assert abs(exact - round(exact)) <= Fraction(1, 10**9) * exact, (g, float(exact))
    # a pilot of one edge: undefined
    s1 = gs.GsSums()
    s1.k, s1.m, s1.mask = 1, m, gs.GS_CONNECTED
    assert all(v is None for v in gs.gs_sample_size(s1, 0.1).values())
