"""Pins of the oracle's Algorithm 7 (micro-level estimation).

At p_e = 1 every neighbour is probed once and the per-edge statistics are
exact; they are checked against brute-force enumeration of every 3- and
4-vertex set containing the edge (tests/brute.py ``edge_roles``): x3, x4, x5
count the 3-sets by type, x7 the 4-cliques, x8 the diamonds whose chord is
the edge, omega the diamonds with the edge on the rim, x9 the tailed
triangles whose pendant edge is the edge, x10 the 4-cycles, x11 the 3-stars,
x12 the 4-paths with the edge in the middle, x13 the pairs (triangle vertex,
vertex adjacent to neither end); x14-x17 follow the printed formulas. Below
p_e = 1 the weighted probes are unbiased: their mean over seeds converges to
the exact values."""
import itertools
import math

import numpy as np
import pytest

import brute
import oracle
import synth


def _random_graphs():
    rng = np.random.default_rng(17)
    for n, p in ((6, 0.5), (8, 0.6), (10, 0.4), (12, 0.5), (12, 0.8), (9, 0.9)):
        for _ in range(4):
            A = np.triu((rng.random((n, n)) < p).astype(np.int64), 1)
            A = A + A.T
            yield A


def _csr(A):
    n = len(A)
    a, b = np.nonzero(np.triu(A, 1))
    return synth.from_pairs(n, a, b)


def test_exact_micro_statistics_equal_brute_force_roles():
    checked = 0
    for A in _random_graphs():
        rp, col = _csr(A)
        n, m = len(A), int(A.sum()) // 2
        pairs = synth.upper_pairs(rp, col)
        if len(pairs) == 0:
            continue
        x, om = oracle.micro(rp, col, pairs, 1.0, seed=3)
        d = A.sum(1)
        for j, (p, q) in enumerate(pairs):
            r = brute.edge_roles(A, int(p), int(q))
            row = dict(zip(oracle.MICRO, x[j]))
            t = r["tri"]
            ab = r["wedge"]
            R = r["lone"]
            assert (row[3], row[4], row[5]) == (t, ab, R)
            assert row[6] == math.comb(n, 3) - t - ab - R
            assert row[7] == r["k4"]
            assert row[8] == r["diamond_chord"]
            assert om[j] == r["diamond_rim"]
            assert row[9] == r["tailed_tail"]
            assert row[10] == r["c4"]
            assert row[11] == r["star"]
            assert row[12] == r["path_mid"]
            assert row[13] == r["tri_far"]
            assert row[14] == ab * R
            assert row[15] == m - (t + d[p] + d[q] + 1) - r["diamond_rim"]
            assert row[16] == math.comb(R, 2)
            assert row[17] == math.comb(n, 4) - sum(row[i] for i in range(7, 17))
            checked += 1
    assert checked > 300


def test_exact_micro_sums_equal_global_counts_times_edge_roles():
    """Summed over every edge, each exact statistic counts every copy of its
    graphlet once per edge in that role: 4-cliques 6 times, diamonds once as
    chord and 4 times on the rim, tailed triangles once as tail, 4-cycles 4
    times, 3-stars 3 times, 4-paths once in the middle."""
    rp, col = synth.chung_lu(400, 3000, 2.1, 80.0, seed=5)
    pairs = synth.upper_pairs(rp, col)
    x, om = oracle.micro(rp, col, pairs, 1.0, seed=1)
    ex = oracle.exact_counts(rp, col)
    s = dict(zip(oracle.MICRO, x.sum(0)))
    assert s[3] == 3 * ex[3]
    assert s[7] == 6 * ex[7]
    assert s[8] == ex[8] and om.sum() == 4 * ex[8]
    assert s[9] == ex[9]
    assert s[10] == 4 * ex[10]
    assert s[11] == 3 * ex[11]
    assert s[12] == ex[12]


def test_sampled_micro_statistics_are_unbiased_and_exact_at_full_probe_rate():
    """p_e = 0.25 on a heavy-tailed graph: over 400 seeds the mean of the
    weighted hit sums (x7, x9, x10, omega) of every edge together converges
    to the exact total (4.5 standard errors); every probe count is at least
    one, so an estimate can only differ from the truth when a window misses."""
    rp, col = synth.chung_lu(300, 2500, 2.1, 60.0, seed=9)
    pairs = synth.explicit_sample(rp, col, 0.3, seed=4)
    exact, om1 = oracle.micro(rp, col, pairs, 1.0, seed=0)
    cols = [oracle.MICRO.index(i) for i in (7, 9, 10)]
    want = np.append(exact[:, cols].sum(0), om1.sum())
    draws = []
    for sd in range(400):
        x, om = oracle.micro(rp, col, pairs, 0.25, seed=sd)
        draws.append(np.append(x[:, cols].sum(0), om.sum()))
        # deterministic columns do not depend on the probes
        assert np.array_equal(x[:, :3], exact[:, :3])
    draws = np.array(draws)
    mean, se = draws.mean(0), draws.std(0, ddof=1) / math.sqrt(len(draws))
    assert np.all(np.abs(mean - want) <= 4.5 * se + 1e-9), (mean, want, se)
    assert np.all(draws.std(0) > 0)  # the probes really were sampled
    # the same seed gives the same estimates
    a, _ = oracle.micro(rp, col, pairs, 0.25, seed=7)
    b, _ = oracle.micro(rp, col, pairs, 0.25, seed=7)
    assert np.array_equal(a, b)


def test_micro_rejects_bad_inputs():
    rp, col = synth.er(30, 60, seed=1)
    pairs = synth.upper_pairs(rp, col)[:3]
    with pytest.raises(ValueError):
        oracle.micro(rp, col, pairs, 0.0)
    with pytest.raises(ValueError):
        oracle.micro(rp, col, pairs, 1.5)
    nz = set(map(tuple, synth.upper_pairs(rp, col)))
    bad = next((0, y) for y in range(1, 30) if (0, y) not in nz)
    with pytest.raises(ValueError):
        oracle.micro(rp, col, np.array([bad], dtype=np.int32))
