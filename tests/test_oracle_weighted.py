"""Pins of the oracle's weighted sampling path (Sec. 3.1's weighted
distribution F with k-core numbers or degrees as weights) and of its
Horvitz-Thompson estimates (sigma_e = 1 / pi_e, Sec. 2.3's inverse sampling
probability per edge).

core numbers: closed forms, the definition evaluated by repeated deletion
on small graphs, and networkx where it is installed.
sampler: with equal weights it draws the uniform sample of the same seed;
each edge's inclusion frequency over seeds matches pi_e.
estimates: exact when every pi_e is 1; unbiased over seeds with a variance
estimate that matches the spread; with equal weights X = sum y / p."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


def _graph(n, edges):
    a, b = zip(*edges) if edges else ((), ())
    return synth.from_pairs(n, np.array(a, dtype=np.int64), np.array(b, dtype=np.int64))


def _cores_by_definition(n, A):
    """core(v) = max k such that v survives repeated deletion of vertices of
    degree < k."""
    core = np.zeros(n, dtype=np.int64)
    for k in range(1, n):
        alive = np.ones(n, dtype=bool)
        changed = True
        while changed:
            deg = (A[:, alive].sum(1)) * alive
            drop = alive & (deg < k)
            changed = drop.any()
            alive &= ~drop
        core[alive] = k
    return core


def test_core_numbers_closed_forms():
    n = 9
    rp, col = _graph(n, list(itertools.combinations(range(n), 2)))
    assert (oracle.core_numbers(rp, col) == n - 1).all()
    rp, col = _graph(10, [(i, (i + 1) % 10) for i in range(10)])
    assert (oracle.core_numbers(rp, col) == 2).all()
    rp, col = _graph(10, [(i, i + 1) for i in range(9)])
    assert (oracle.core_numbers(rp, col) == 1).all()
    rp, col = _graph(8, [(0, i) for i in range(1, 8)])
    assert (oracle.core_numbers(rp, col) == 1).all()
    rp, col = _graph(9, [(i, 4 + j) for i in range(4) for j in range(5)])
    assert (oracle.core_numbers(rp, col) == 4).all()
    petersen = [(i, (i + 1) % 5) for i in range(5)] + [(5 + i, 5 + (i + 2) % 5)
                                                       for i in range(5)] + [(i, i + 5)
                                                                             for i in range(5)]
    rp, col = _graph(10, petersen)
    assert (oracle.core_numbers(rp, col) == 3).all()
    rp, col = _graph(5, [])
    assert (oracle.core_numbers(rp, col) == 0).all()


def test_core_numbers_equal_the_definition_on_random_graphs():
    rng = np.random.default_rng(5)
    for n, p in ((8, 0.3), (12, 0.4), (15, 0.5), (20, 0.25), (16, 0.7)):
        A = np.triu((rng.random((n, n)) < p).astype(np.int64), 1)
        A = A + A.T
        rp, col = _graph(n, list(zip(*np.nonzero(np.triu(A, 1)))))
        assert np.array_equal(oracle.core_numbers(rp, col), _cores_by_definition(n, A))


def test_core_numbers_equal_networkx():
    nx = pytest.importorskip("networkx")
    rp, col = synth.chung_lu(3000, 20000, 2.1, 300.0, seed=2)
    G = nx.Graph()
    G.add_nodes_from(range(len(rp) - 1))
    pairs = synth.upper_pairs(rp, col)
    G.add_edges_from(map(tuple, pairs.tolist()))
    want = nx.core_number(G)
    got = oracle.core_numbers(rp, col)
    assert all(got[v] == want[v] for v in range(len(rp) - 1))


def test_equal_weights_draw_the_uniform_sample():
    rp, col = synth.er(800, 6000, seed=3)
    ones = np.ones(len(rp) - 1, dtype=np.int32)
    for frac, seed in ((0.1, 1), (0.37, 2), (1.0, 3)):
        pairs, w, s = oracle.sample_weighted(rp, col, ones * 5, frac, seed)
        assert np.array_equal(pairs, oracle.sample(rp, col, frac, seed))
        assert (w == 5).all()


def test_inclusion_frequency_matches_pi():
    rp, col = synth.chung_lu(300, 1500, 2.1, 40.0, seed=8)
    core = oracle.core_numbers(rp, col)
    up = synth.upper_pairs(rp, col)
    we = np.minimum(core[up[:, 0]], core[up[:, 1]])
    _, _, s = oracle.sample_weighted(rp, col, core, 0.2, 0)
    pi = np.minimum(1.0, s * we)
    keys = up[:, 0].astype(np.int64) * (len(rp) - 1) + up[:, 1]
    hits = np.zeros(len(up))
    trials = 2000
    for sd in range(trials):
        pairs, _, _ = oracle.sample_weighted(rp, col, core, 0.2, sd)
        hits[np.searchsorted(keys, pairs[:, 0].astype(np.int64) * (len(rp) - 1) + pairs[:, 1])] += 1
    freq = hits / trials
    se = np.sqrt(pi * (1 - pi) / trials)
    assert np.all(np.abs(freq - pi) <= 5 * se + 1e-12)
    # the expected sample size is fraction * M (no weight reaches pi = 1 here)
    assert pi.max() < 1.0 and abs(pi.sum() - 0.2 * len(up)) < 1e-6 * len(up)


def test_ht_estimate_is_exact_when_every_edge_is_kept():
    rp, col = synth.chung_lu(500, 3000, 2.1, 60.0, seed=4)
    big = np.full(len(rp) - 1, 1000, dtype=np.int32)
    pairs, w, s = oracle.sample_weighted(rp, col, big, 1.0, 1)  # equal weights: pi = 1
    assert len(pairs) == len(col) // 2
    lc = oracle.local_counts(rp, col, pairs)
    res = oracle.ht_estimate(lc, w, s, len(col) // 2)
    exact = oracle.exact_counts(rp, col)
    for g in oracle.GRAPHLETS:
        assert res[g]["exact"] == exact[g] and res[g]["X"] == exact[g] and res[g]["V"] == 0.0


def test_ht_estimate_with_equal_weights_is_the_inverse_probability_sum():
    rp, col = synth.er(400, 4000, seed=6)
    ones = np.ones(len(rp) - 1, dtype=np.int32)
    pairs, w, s = oracle.sample_weighted(rp, col, ones, 0.25, 9)
    lc = oracle.local_counts(rp, col, pairs)
    res = oracle.ht_estimate(lc, w, s, len(col) // 2)
    _, _, nmat = oracle.numerators(lc, per_edge=True)
    p = min(1.0, s)
    for i, g in enumerate(oracle.GRAPHLETS):
        direct = float(nmat[:, i].sum()) / (oracle.DENOM[g] * p)
        assert res[g]["X"] == pytest.approx(direct, rel=1e-12)


def test_ht_estimate_is_unbiased_with_matching_variance():
    """k-core weights on a power-law graph: over 600 seeds the mean of X is
    within 4.5 standard errors of the exact count and the mean variance
    estimate matches the spread of X."""
    rp, col = synth.chung_lu(600, 4000, 2.1, 80.0, seed=10)
    m = len(col) // 2
    core = oracle.core_numbers(rp, col)
    exact = oracle.exact_counts(rp, col)
    up = synth.upper_pairs(rp, col)
    lc_all = oracle.local_counts(rp, col, up)
    n_v = len(rp) - 1
    keys = up[:, 0].astype(np.int64) * n_v + up[:, 1]
    xs = {g: [] for g in oracle.GRAPHLETS}
    vs = {g: [] for g in oracle.GRAPHLETS}
    for sd in range(600):
        pairs, w, s = oracle.sample_weighted(rp, col, core, 0.15, sd)
        idx = np.searchsorted(keys, pairs[:, 0].astype(np.int64) * n_v + pairs[:, 1])
        lc = {k: v[idx] for k, v in lc_all.items()}
        res = oracle.ht_estimate(lc, w, s, m)
        for g in oracle.GRAPHLETS:
            xs[g].append(res[g]["X"])
            vs[g].append(res[g]["V"])
    for g in oracle.GRAPHLETS:
        mean = float(np.mean(xs[g]))
        se = math.sqrt(float(np.var(xs[g], ddof=1)) / len(xs[g]))
        assert abs(mean - exact[g]) <= 4.5 * se + 1e-9, (g, mean, exact[g], se)
        if exact[g] >= 1000:
            ratio = float(np.var(xs[g], ddof=1)) / float(np.mean(vs[g]))
            assert 0.7 < ratio < 1.4, (g, ratio)
