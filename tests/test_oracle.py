"""Pins for the CPU oracle: each check comes from something other than the
oracle itself (Table 1, brute-force enumeration, closed forms, counting
identities, a published RNG test vector, statistics)."""
import itertools
import math

import numpy as np
import pytest

import brute
import oracle
import synth

CONNECTED = (3, 4, 7, 8, 9, 10, 11, 12)


def oracle_exact(row_ptr, col):
    return oracle.exact_counts(row_ptr, col)


# ------------------------------------------------------------------ Table 1

def test_table1_properties_of_graphlet_definitions():
    """The edge lists used to build graphlets reproduce Table 1's columns."""
    table = brute.load_table1()
    for gid, (n, edges) in brute.GRAPHLET_EDGES.items():
        got = brute.properties(n, edges)
        want = table[gid]
        assert got["n"] == want["n"], gid
        assert round(got["rho"], 2) == pytest.approx(want["rho"], abs=0.006), gid
        assert got["dmax"] == want["dmax"], gid
        assert got["dbar"] == pytest.approx(want["dbar"], abs=0.006), gid
        for key in ("tri", "core", "chi", "diam", "comp"):
            assert got[key] == want[key], (gid, key)


@pytest.mark.parametrize("gid", [3, 4, 7, 8, 9, 10, 11, 12])
def test_each_connected_graphlet_counts_itself_once(gid):
    n, edges = brute.GRAPHLET_EDGES[gid]
    rp, col = brute.csr_from_edges(n, edges)
    got = oracle_exact(rp, col)
    want = brute.brute_counts(brute.adjacency(n, edges))
    assert got[gid] == 1
    for g in CONNECTED:
        assert got[g] == want[g], g
    if n == 4:
        for g in (7, 8, 9, 10, 11, 12):
            assert got[g] == (1 if g == gid else 0)


# ------------------------------------------------------------------ brute force

def _check_against_brute(A):
    rp, col = brute.csr_from_adjacency(A)
    if len(col) == 0:
        return
    got = oracle_exact(rp, col)
    want = brute.brute_counts(A)
    for g in CONNECTED:
        assert got[g] == want[g], (g, got, want)


def test_all_labelled_graphs_on_five_vertices():
    pairs = list(itertools.combinations(range(5), 2))
    for mask in range(1 << len(pairs)):
        A = np.zeros((5, 5), dtype=np.int64)
        for i, (a, b) in enumerate(pairs):
            if mask >> i & 1:
                A[a, b] = A[b, a] = 1
        _check_against_brute(A)


def test_random_labelled_graphs_on_six_vertices():
    pairs = list(itertools.combinations(range(6), 2))
    rng = np.random.default_rng(6)
    for mask in rng.choice(1 << len(pairs), size=400, replace=False):
        A = np.zeros((6, 6), dtype=np.int64)
        for i, (a, b) in enumerate(pairs):
            if int(mask) >> i & 1:
                A[a, b] = A[b, a] = 1
        _check_against_brute(A)


@pytest.mark.parametrize("n,p,seed", [(8, 0.5, 1), (10, 0.3, 2), (10, 0.7, 3), (12, 0.4, 4),
                                      (12, 0.6, 5), (12, 0.9, 6), (11, 0.2, 7)])
def test_random_gnp_against_brute_force(n, p, seed):
    rng = np.random.default_rng(seed)
    U = np.triu(rng.random((n, n)) < p, 1)
    A = (U | U.T).astype(np.int64)
    _check_against_brute(A)


def test_literal_algorithm4_disagrees_with_brute_force():
    """Algorithm 4 as printed (testing lambda_2) counts the wrong thing; the
    reading used by the oracle (testing S_v membership) is the one that
    matches enumeration.  This is the planted mistake for the cycle count."""
    rng = np.random.default_rng(11)
    mismatches = 0
    for trial in range(20):
        n = 9
        U = np.triu(rng.random((n, n)) < 0.45, 1)
        A = (U | U.T).astype(np.int64)
        rp, col = brute.csr_from_adjacency(A)
        pairs = synth.upper_pairs(rp, col)
        if len(pairs) == 0:
            continue
        lit = oracle.local_counts(rp, col, pairs, _literal_alg4=True)
        ok = oracle.local_counts(rp, col, pairs)
        s_lit, _ = oracle.numerators(lit)
        s_ok, _ = oracle.numerators(ok)
        want = brute.brute_counts(A)
        assert s_ok[10] == 4 * want[10]
        mismatches += s_lit[10] != 4 * want[10]
    assert mismatches > 0


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("kind,args", [
    ("complete", (4,)), ("complete", (5,)), ("complete", (7,)), ("complete", (9,)),
    ("cycle", (3,)), ("cycle", (4,)), ("cycle", (5,)), ("cycle", (9,)), ("cycle", (40,)),
    ("path", (2,)), ("path", (3,)), ("path", (4,)), ("path", (30,)),
    ("star", (1,)), ("star", (2,)), ("star", (5,)), ("star", (40,)),
    ("bipartite", (1, 1)), ("bipartite", (2, 2)), ("bipartite", (3, 4)), ("bipartite", (6, 9)),
])
def test_closed_forms(kind, args):
    n, edges = brute.family_edges(kind, *args)
    rp, col = brute.csr_from_edges(n, edges)
    got = oracle_exact(rp, col)
    want = brute.closed_form(kind, *args)
    for g in CONNECTED:
        assert got[g] == want[g], (kind, args, g)


# ------------------------------------------------------------------ identities

@pytest.mark.parametrize("maker", [
    lambda: synth.er(120, 900, seed=5),
    lambda: synth.chung_lu(400, 3000, 2.1, 150.0, seed=9),
    lambda: synth.rgg(300, 0.12, seed=3),
    lambda: synth.rmat(9, 8, seed=4),
])
def test_counting_identities(maker):
    rp, col = maker()
    c = oracle_exact(rp, col)
    ids = brute.identities(rp, col)
    assert ids["wedges"] == c[4] + 3 * c[3]
    assert ids["claws"] == c[11] + c[9] + 2 * c[8] + 4 * c[7]
    assert ids["paths3_raw"] - 3 * c[3] == c[12] + 2 * c[9] + 4 * c[10] + 6 * c[8] + 12 * c[7]
    A = brute.adjacency_from_csr(rp, col)
    A2 = A @ A
    assert int(np.trace(A2 @ A)) == 6 * c[3]
    tr4 = int(np.sum(A2 * A2))  # tr(A^4) = ||A^2||_F^2 for symmetric A
    assert tr4 - 2 * ids["sum_d2"] + 2 * ids["M"] == 8 * (c[10] + c[8] + 3 * c[7])


def test_triangle_sum_over_edges_is_three_per_triangle():
    rp, col = synth.er(200, 2500, seed=8)
    pairs = synth.upper_pairs(rp, col)
    lc = oracle.local_counts(rp, col, pairs, four=False)
    A = brute.adjacency_from_csr(rp, col)
    assert int(lc["t"].sum()) == int(np.trace(A @ A @ A)) // 6 * 3
    d = np.diff(rp)
    # a + b + 2 t = d_u + d_v - 2 per edge
    du, dv = d[pairs[:, 0]], d[pairs[:, 1]]
    assert np.array_equal(lc["a"] + lc["b"] + 2 * lc["t"], du + dv - 2)


def test_orientation_and_order_do_not_change_counts():
    rp, col = synth.er(150, 1200, seed=12)
    pairs = synth.upper_pairs(rp, col)
    base = oracle.local_counts(rp, col, pairs)
    rng = np.random.default_rng(1)
    perm = rng.permutation(len(pairs))
    flipped = pairs[perm][:, ::-1].copy()
    other = oracle.local_counts(rp, col, flipped)
    for key in ("t", "k", "q"):
        assert np.array_equal(base[key][perm], other[key])
    assert np.array_equal((base["a"] + base["b"])[perm], other["a"] + other["b"])


# ------------------------------------------------------------------ sampler

def test_splitmix64_published_vector():
    """SplitMix64 seeded with 1234567: the first five outputs published with
    the reference generator's test suite."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    state = 1234567
    got = []
    for _ in range(5):
        got.append(oracle.splitmix64(state))
        state = (state + 0x9E3779B97F4A7C15) % 2**64
    assert got == want


def test_sampler_limits_and_nesting():
    rp, col = synth.er(300, 4000, seed=2)
    allp = synth.upper_pairs(rp, col)
    assert np.array_equal(oracle.sample(rp, col, 1.0, 7), allp)
    assert len(oracle.sample(rp, col, 0.0, 7)) == 0
    a = oracle.sample(rp, col, 0.1, 99)
    b = oracle.sample(rp, col, 0.3, 99)
    sa = {tuple(x) for x in a}
    sb = {tuple(x) for x in b}
    assert sa <= sb
    assert np.array_equal(a, oracle.sample(rp, col, 0.1, 99))
    assert not np.array_equal(a, oracle.sample(rp, col, 0.1, 100))


def test_sampler_rate_is_binomial():
    rp, col = synth.er(2000, 20000, seed=1)
    m = len(col) // 2
    for p in (0.01, 0.1, 0.5):
        k = len(oracle.sample(rp, col, p, 12345))
        sd = math.sqrt(m * p * (1 - p))
        assert abs(k - m * p) < 5 * sd


# ------------------------------------------------------------------ estimator

def test_full_sample_gives_exact_counts_and_zero_variance():
    rp, col = synth.er(100, 700, seed=21)
    pairs = synth.upper_pairs(rp, col)
    res = oracle.count_estimate(rp, col, pairs)
    A = brute.adjacency_from_csr(rp, col)
    want = brute.brute_counts(A)
    for g in CONNECTED:
        e = res["est"][g]
        assert e["exact"] == want[g]
        assert e["X"] == float(want[g])
        assert e["V"] == 0.0
        assert e["lb"] == e["ub"] == e["X"]


def test_variance_matches_two_pass_sample_variance():
    rp, col = synth.chung_lu(2000, 15000, 2.1, 300.0, seed=4)
    m = len(col) // 2
    pairs = oracle.sample(rp, col, 0.05, 3)
    lc = oracle.local_counts(rp, col, pairs)
    s, s2, nmat = oracle.numerators(lc, per_edge=True)
    est = oracle.estimate(s, s2, m, len(pairs))
    k = len(pairs)
    for i, g in enumerate(oracle.GRAPHLETS):
        y = nmat[:, i].astype(np.float64) / oracle.DENOM[g]
        x_direct = m * y.mean()
        v_direct = m * m * (1 - k / m) * y.var(ddof=1) / k
        assert est[g]["X"] == pytest.approx(x_direct, rel=1e-12)
        assert est[g]["V"] == pytest.approx(v_direct, rel=1e-9, abs=1e-9)


def test_unbiased_and_covering_over_seeds():
    """Mean of X over seeds approaches the exact count (unbiasedness,
    Sec. 2.4) and the 95% interval covers it about 95% of the time
    (Sec. 6.2): with 2000 seeds the coverage of every graphlet with at least
    1000 copies lies within 95% +- 3 points (six binomial standard
    deviations)."""
    rp, col = synth.er(400, 8000, seed=31)
    m = len(col) // 2
    exact = oracle_exact(rp, col)
    pairs_all = synth.upper_pairs(rp, col)
    lc_all = oracle.local_counts(rp, col, pairs_all)
    seeds = range(2000)
    xs = {g: [] for g in CONNECTED}
    cover = {g: 0 for g in CONNECTED}
    vs = {g: [] for g in CONNECTED}
    n_v = len(rp) - 1
    keys_all = pairs_all[:, 0].astype(np.int64) * n_v + pairs_all[:, 1]
    for sd in seeds:
        smp = oracle.sample(rp, col, 0.1, sd)
        idx = np.searchsorted(keys_all, smp[:, 0].astype(np.int64) * n_v + smp[:, 1])
        sub = {key: val[idx] for key, val in lc_all.items()}
        s, s2 = oracle.numerators(sub)
        est = oracle.estimate(s, s2, m, len(idx))
        for g in CONNECTED:
            xs[g].append(est[g]["X"])
            vs[g].append(est[g]["V"])
            cover[g] += est[g]["lb"] <= exact[g] <= est[g]["ub"]
    n = len(seeds)
    for g in CONNECTED:
        mean = float(np.mean(xs[g]))
        se = math.sqrt(float(np.mean(vs[g])) / n)
        assert abs(mean - exact[g]) <= 4.5 * se + 1e-9, (g, mean, exact[g], se)
        if exact[g] >= 1000:
            assert 0.92 * n <= cover[g] <= 0.98 * n, (g, cover[g])
        emp = float(np.var(xs[g], ddof=1))
        if exact[g] >= 1000:
            assert 0.6 < emp / float(np.mean(vs[g])) < 1.6, g


# ------------------------------------------------------------------ disconnected graphlets

DISC = oracle.DISCONNECTED


def _disc_exact(rp, col):
    return {g: r["exact"] for g, r in
            oracle.disconnected_estimate(rp, col, synth.upper_pairs(rp, col)).items()}


@pytest.mark.parametrize("seed", range(8))
def test_disconnected_exact_counts_match_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(12):
        n = int(rng.integers(4, 12))
        A = np.triu((rng.random((n, n)) < rng.random()).astype(np.int64), 1)
        A = A + A.T
        if A.sum() == 0:
            continue
        rp, col = brute.csr_from_adjacency(A)
        want = brute.brute_counts(A)
        got = _disc_exact(rp, col)
        for g in DISC:
            assert got[g] == want[g], (g, got[g], want[g])


def test_disconnected_closed_forms():
    # one edge on n vertices: every other vertex is isolated
    for n in (4, 7, 30):
        rp, col = synth.from_pairs(n, np.array([0]), np.array([1]))
        got = _disc_exact(rp, col)
        assert got[5] == n - 2 and got[6] == math.comb(n, 3) - (n - 2)
        assert got[16] == math.comb(n - 2, 2)
        assert got[17] == math.comb(n, 4) - math.comb(n - 2, 2)
        assert got[13] == got[14] == got[15] == 0
    # K_n has no disconnected induced subgraph
    n, edges = brute.family_edges("complete", 9)
    rp, col = synth.from_pairs(n, np.array([e[0] for e in edges]), np.array([e[1] for e in edges]))
    assert all(v == 0 for v in _disc_exact(rp, col).values())
    # a perfect matching on 2p vertices: pairs of matching edges are G15,
    # an edge with two vertices of other edges is G16
    p = 6
    rp, col = synth.from_pairs(2 * p, np.arange(0, 2 * p, 2), np.arange(1, 2 * p, 2))
    got = _disc_exact(rp, col)
    assert got[15] == math.comb(p, 2)
    assert got[16] == p * (math.comb(2 * p - 2, 2) - (p - 1))
    assert got[5] == p * (2 * p - 2) and got[13] == got[14] == 0


def test_printed_disconnected_block_disagrees_with_brute_force():
    """As printed, the estimators of G13 and G14 use C13 and C14 the other
    way round; that reading fails brute force (the corrected one passes in
    the tests above)."""
    rng = np.random.default_rng(7)
    disagree = 0
    for _ in range(30):
        n = int(rng.integers(5, 10))
        A = np.triu((rng.random((n, n)) < 0.5).astype(np.int64), 1)
        A = A + A.T
        if A.sum() == 0:
            continue
        rp, col = brute.csr_from_adjacency(A)
        pairs = synth.upper_pairs(rp, col)
        lc = oracle.local_counts(rp, col, pairs)
        R = (n - 2 - lc["t"] - lc["a"] - lc["b"]).astype(object)
        c13 = int(np.sum((lc["a"] + lc["b"]).astype(object) * R))  # (a+b) R
        x9 = oracle.exact_counts(rp, col)[9]
        literal_13 = (c13 - x9) / 3  # printed: C13 where C14 = sum t R belongs
        if literal_13 != brute.brute_counts(A)[13]:
            disagree += 1
    assert disagree >= 20


def test_disconnected_unbiased_over_seeds():
    rp, col = synth.er(300, 3000, seed=5)
    exact = _disc_exact(rp, col)
    xs = {g: [] for g in DISC}
    vs = {g: [] for g in DISC}
    for sd in range(120):
        est = oracle.disconnected_estimate(rp, col, oracle.sample(rp, col, 0.1, sd))
        for g in DISC:
            xs[g].append(est[g]["X"])
            vs[g].append(est[g]["V"])
    for g in DISC:
        mean = float(np.mean(xs[g]))
        se = math.sqrt(float(np.mean(vs[g])) / len(xs[g]))
        assert abs(mean - exact[g]) <= 4.5 * se + 1e-6 * abs(exact[g]) + 1e-9, (g, mean, exact[g])


# ------------------------------------------------------------------ Algorithm 8 (adaptive)

def test_adaptive_with_zero_beta_runs_t_max_halving_phi():
    """beta = 0 runs t_max iterations; iteration t draws ceil(phi_t (M - |J|))
    new edges with phi halving after each draw."""
    rp, col = synth.er_2000()
    m = len(col) // 2
    r = oracle.adaptive_estimate(rp, col, 0.0, 6, 0.05, 3)
    assert r["iters"] == 6
    J, phi = 0, 0.05
    for _ in range(6):
        J, phi = min(m, J + math.ceil(phi * (m - J))), phi / 2
    assert r["K"] == J and r["p"] == J / m


def test_adaptive_result_is_the_fixed_size_sample_and_larger_beta_stops_no_later():
    rp, col = synth.chung_lu(3000, 20000, 2.1, 300.0, seed=8)
    prev_iters = None
    for beta in (0.001, 0.01, 0.1):
        r = oracle.adaptive_estimate(rp, col, beta, 10, 0.02, 5)
        pairs = oracle.sample_fixed(rp, col, r["K"], 5)
        s, s2 = oracle.numerators(oracle.local_counts(rp, col, pairs))
        assert s == r["sums"] and s2 == r["sq"]
        if prev_iters is not None:
            assert r["iters"] <= prev_iters
        prev_iters = r["iters"]


def _union_graph(spec):
    """Disjoint union of small components; returns CSR and the vertex range
    end of each component kind, in order."""
    a, b, ends, n = [], [], [], 0
    for kind, copies in spec:
        for _ in range(copies):
            if kind == "K4":
                for i in range(4):
                    for j in range(i + 1, 4):
                        a.append(n + i)
                        b.append(n + j)
                n += 4
            elif kind == "P3":
                a += [n, n + 1]
                b += [n + 1, n + 2]
                n += 3
        ends.append((kind, n))
    rp, col = synth.from_pairs(n, np.array(a), np.array(b))
    return rp, col, ends


def _closed_form_graph(kind):
    """Edge-transitive graphs with their closed-form connected counts."""
    if kind == "cycle30":
        n = 30
        rp, col = synth.from_pairs(n, np.arange(n), (np.arange(n) + 1) % n)
        return rp, col, {4: n, 12: n}
    if kind == "K12":
        n = 12
        a, b = zip(*itertools.combinations(range(n), 2))
        rp, col = synth.from_pairs(n, np.array(a), np.array(b))
        return rp, col, {3: math.comb(n, 3), 7: math.comb(n, 4)}
    if kind == "K4_6":
        p, q = 4, 6
        a = [i for i in range(p) for _ in range(q)]
        b = [p + j for _ in range(p) for j in range(q)]
        rp, col = synth.from_pairs(p + q, np.array(a), np.array(b))
        return rp, col, {4: p * math.comb(q, 2) + q * math.comb(p, 2),
                         10: math.comb(p, 2) * math.comb(q, 2),
                         11: p * math.comb(q, 3) + q * math.comb(p, 3)}
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["cycle30", "K12", "K4_6"])
@pytest.mark.parametrize("beta", [0.0, 0.25])
def test_adaptive_stops_at_the_second_iteration_on_edge_transitive_graphs(kind, beta):
    """Every edge of an edge-transitive graph has the same (t, a, b, k, q), so
    any non-empty sample estimates every count exactly (sigma K N / D = M N /
    D): the first iteration (at least one edge) already gives the closed
    form, the second changes nothing (loss 0 <= beta, also beta = 0) and the
    loop stops there."""
    rp, col, closed = _closed_form_graph(kind)
    m = len(col) // 2
    for seed in (1, 2, 3):
        r = oracle.adaptive_estimate(rp, col, beta, 20, 0.3, seed)
        assert r["iters"] == 2, (kind, seed, r["iters"])
        for g in oracle.GRAPHLETS:
            assert r["est"][g]["X"] == float(closed.get(g, 0)), (kind, g)
        k1 = math.ceil(0.3 * m)
        assert r["K"] == min(m, k1 + math.ceil(0.15 * (m - k1)))


def test_adaptive_loss_sequence_on_a_two_class_graph():
    """30 copies of K4 and 2 of the path P3, seed 11, beta 0.02, phi 0.1;
    iteration t adds the next ceil(phi_t (M - |J|)) edges in sampler-key
    order.
    Per-edge numerators by hand: a K4 edge has t = 2, a = b = 0, k = 1, so
    N3 = 2, N7 = 1 and every other N is 0; a P3 edge has t = 0, a + b = 1, so
    N4 = 1 and every 4-node N is 0. With n_K, n_P edges of each kind in the
    nested sample (K = n_K + n_P, M = 184): X7 = M n_K / (6 K),
    X4 = M n_P / (2 K), X3 = M 2 n_K / (3 K), other 4-node X = 0. The loss of
    iteration t is max over G^(4) of |X^(t) - X^(t-1)| / |X^(t-1)|, i.e.
    only X7 moves. The schedule stops at iteration 3; taking the maximum
    over every graphlet (X4 jumps from 0 when a P3 edge enters), an absolute
    instead of a relative change, or comparing with X^(t-2) would stop
    later, as the replay below shows."""
    rp, col, ends = _union_graph([("K4", 30), ("P3", 2)])
    m = len(col) // 2
    assert m == 184
    k4_end = ends[0][1]

    up = synth.upper_pairs(rp, col)

    def replay(rule, beta=0.02, phi=0.1, seed=11, t_max=12):
        keys = oracle.sample_keys(rp, col, seed)
        order = np.lexsort((np.arange(m), keys))
        J, t, loss, hist = 0, 0, 1.0, []
        while loss > beta and t < t_max:
            J = min(m, J + math.ceil(phi * (m - J)))
            u = up[np.sort(order[:J])][:, 0]
            nk, npath = int((u < k4_end).sum()), int((u >= k4_end).sum())
            k = nk + npath
            x = {3: m * 2 * nk / (3 * k), 4: m * npath / (2 * k), 7: m * nk / (6 * k)}
            ref = hist[-2] if rule == "t-2" and len(hist) >= 2 else (hist[-1] if hist else None)
            if ref is None:
                loss = 1.0
            else:
                keys_ = (3, 4, 7) if rule == "all" else (7,)
                changes = []
                for g in keys_:
                    if x[g] == ref[g]:
                        changes.append(0.0)
                    elif ref[g] == 0:
                        changes.append(math.inf)
                    else:
                        d = abs(x[g] - ref[g])
                        changes.append(d if rule == "abs" else d / abs(ref[g]))
                loss = max(changes)
            hist.append(x)
            phi, t = phi / 2, t + 1
        return t, J

    want = replay("paper")
    assert want[0] == 3
    for other in ("all", "abs", "t-2"):
        assert replay(other)[0] != want[0], other
    r = oracle.adaptive_estimate(rp, col, 0.02, 12, 0.1, 11)
    assert (r["iters"], r["K"]) == want


def test_adaptive_loss_helpers():
    assert oracle.adaptive_loss_graphlets(oracle.GRAPHLETS) == (7, 8, 9, 10, 11, 12)
    assert oracle.adaptive_loss_graphlets((3, 4)) == (3, 4)
    assert oracle.adaptive_loss_graphlets((3, 10)) == (10,)
    assert oracle.relative_change(0.0, 0.0) == 0.0
    assert oracle.relative_change(1.0, 0.0) == math.inf
    assert oracle.relative_change(90.0, 100.0) == 0.1
    assert oracle.relative_change(-110.0, -100.0) == 0.1


def test_oracle_pool_returns_the_oracle_per_edge_output_in_order():
    from oracle_pool import OraclePool
    rp, col = synth.chung_lu(3000, 20000, 2.1, 300.0, seed=12)
    pairs = synth.explicit_sample(rp, col, 0.3, seed=2)
    want = oracle.local_counts(rp, col, pairs)
    with OraclePool(rp, col, workers=2) as pool:
        got = pool.local_counts(pairs)
        got3 = pool.local_counts(pairs[:100], four=False)
    for x in ("t", "a", "b", "k", "q"):
        assert np.array_equal(got[x], want[x]), x
    assert np.array_equal(got3["t"], want["t"][:100])


def test_fixed_size_sample_is_the_smallest_keys_and_nested_with_bernoulli():
    """The keys restated in Python integers agree with the C sampler (each
    Bernoulli sample is the set of keys below its threshold); a fixed-size
    sample has exactly k distinct edges, is nested in k, and lies between
    the Bernoulli samples whose sizes bracket it."""
    rp, col = synth.er(500, 3000, seed=4)
    m = len(col) // 2
    keys = oracle.sample_keys(rp, col, 9)
    up = synth.upper_pairs(rp, col)
    for frac in (0.05, 0.3):
        want = up[keys < int(math.floor(frac * 2.0**53))]
        assert np.array_equal(want, oracle.sample(rp, col, frac, 9))
    prev = set()
    for k in (0, 1, 17, 300, 1500, m):
        smp = oracle.sample_fixed(rp, col, k, 9)
        cur = set(map(tuple, smp.tolist()))
        assert len(smp) == k == len(cur) and prev <= cur
        prev = cur
    small = set(map(tuple, oracle.sample(rp, col, 0.1, 9).tolist()))
    big = set(map(tuple, oracle.sample(rp, col, 0.2, 9).tolist()))
    mid = set(map(tuple, oracle.sample_fixed(rp, col, (len(small) + len(big)) // 2, 9).tolist()))
    assert small <= mid <= big


def test_fixed_size_sample_is_uniform():
    """Each edge's inclusion frequency over seeds is k / M."""
    rp, col = synth.er(60, 200, seed=2)
    m = len(col) // 2
    up = synth.upper_pairs(rp, col)
    keyv = up[:, 0].astype(np.int64) * 60 + up[:, 1]
    hits = np.zeros(m)
    trials = 3000
    for sd in range(trials):
        smp = oracle.sample_fixed(rp, col, 50, sd)
        hits[np.searchsorted(keyv, smp[:, 0].astype(np.int64) * 60 + smp[:, 1])] += 1
    p = 50 / m
    se = math.sqrt(p * (1 - p) / trials)
    assert np.all(np.abs(hits / trials - p) <= 5 * se)
