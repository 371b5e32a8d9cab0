"""Host side of the disconnected graphlets (no GPU): the per-edge numerators
documented in include/graphlet.h, summed exactly and passed through the
library's host estimator, reproduce the oracle's reading of Sec. 2.3 (which
takes the paper's route: C sums and the X equations); shard sums merge
exactly."""
import math

import numpy as np
import pytest

import brute
import oracle
import synth

import paper_1701_01772_gb300 as gs


def _numerators(rp, col, pairs):
    """The seven numerators per edge as documented in include/graphlet.h."""
    n, m = len(rp) - 1, len(col) // 2
    lc = oracle.local_counts(rp, col, pairs)
    rows = []
    for t, a, b, k, q in zip(*(lc[x].tolist() for x in ("t", "a", "b", "k", "q"))):
        n8 = t * (t - 1) // 2 - k
        n9 = t * (a + b) - 4 * n8
        n11 = 2 * (a * (a - 1) // 2 + b * (b - 1) // 2) - t * (a + b) + 4 * n8
        n12 = a * b - q
        R = n - 2 - t - a - b
        c16 = m - (a + t + 1) - (b + t + 1) + 1
        n13 = 2 * t * R - n9
        n14 = (a + b) * R - 2 * n12
        n15 = c16 - k - 4 * n8 - n9 - q - 2 * n12
        n16 = R * (R - 1) // 2 - n15
        n17 = (2 * k + 12 * n8 + 6 * n9 + 3 * q + 2 * n11 + 12 * n12 + 2 * n13 + 6 * n14
               + 6 * n15 + 12 * n16)
        rows.append({5: R, 6: 2 * t + 3 * (a + b) + 6 * R, 13: n13, 14: n14, 15: n15,
                     16: n16, 17: n17})
    return rows


def _sums(rp, col, pairs):
    rows = _numerators(rp, col, pairs)
    s = {g: sum(r[g] for r in rows) for g in gs.DISCONNECTED}
    s2 = {g: sum(r[g] * r[g] for r in rows) for g in gs.DISCONNECTED}
    return gs.disc_sums_from_ints(len(pairs), len(col) // 2, len(rp) - 1, s, s2)


def _agree(got, want):
    for gid in gs.DISCONNECTED:
        for key in ("X", "V"):
            a, b = got[gid][key], want[gid][key]
            if math.isnan(a) or math.isnan(b):
                assert math.isnan(a) and math.isnan(b), (gid, key)
            else:
                assert abs(a - b) <= 1e-12 * max(abs(a), abs(b), 1.0), (gid, key, a, b)
        assert got[gid]["exact"] == want[gid]["exact"], gid


def test_host_estimator_on_documented_numerators_reproduces_the_oracle():
    gs.build()
    cases = [synth.er(300, 3000, seed=5), synth.chung_lu(2000, 15000, 2.1, 300.0, seed=4)]
    for rp, col in cases:
        for pairs in (synth.upper_pairs(rp, col), oracle.sample(rp, col, 0.1, 9)):
            got = gs.gs_estimate_disconnected(_sums(rp, col, pairs)).as_dict()
            _agree(got, oracle.disconnected_estimate(rp, col, pairs))


def test_host_estimator_exact_counts_match_brute_force():
    gs.build()
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(4, 11))
        A = np.triu((rng.random((n, n)) < rng.random()).astype(np.int64), 1)
        A = A + A.T
        if A.sum() == 0:
            continue
        rp, col = brute.csr_from_adjacency(A)
        got = gs.gs_estimate_disconnected(_sums(rp, col, synth.upper_pairs(rp, col))).as_dict()
        want = brute.brute_counts(A)
        for gid in gs.DISCONNECTED:
            assert got[gid]["exact"] == want[gid], gid


def test_disconnected_shard_sums_merge_exactly():
    gs.build()
    rp, col = synth.er(300, 3000, seed=8)
    pairs = oracle.sample(rp, col, 0.3, 2)
    cut = len(pairs) // 3
    merged = gs.gs_sums_disc_merge(_sums(rp, col, pairs[:cut]), _sums(rp, col, pairs[cut:]))
    whole = _sums(rp, col, pairs)
    assert merged.k == whole.k and merged.sums() == whole.sums()
    _agree(gs.gs_estimate_disconnected(merged).as_dict(),
           gs.gs_estimate_disconnected(whole).as_dict())
    other = gs.disc_sums_from_ints(1, whole.m, whole.n + 1, {}, {})
    with pytest.raises(gs.GraphletError):
        gs.gs_sums_disc_merge(whole, other)
