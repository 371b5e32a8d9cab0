"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs. Integer sums and per-edge counts are bit-exact; FP64
estimates agree within 1e-12 relative."""
import itertools

import numpy as np
import pytest

import brute
import oracle
import synth
from gpu_util import assert_estimates_close, assert_sums_equal, oracle_sums, per_edge_reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402

ALL = gs.GRAPHLETS


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    yield


def _graph(rp, col, **kw):
    return gs.Graph.from_numpy(rp, col, **kw)


NO_HUBS = 1  # a 1-byte hub budget disables bitmaps and the co-degree table


def _full_check(rp, col, pairs, mask=gs.GS_CONNECTED, ids=ALL, hub_budget=0, dense_slots=None):
    g = _graph(rp, col, hub_budget_bytes=hub_budget)
    if dense_slots is not None:
        g.ws.set_dense_slots(dense_slots)
    per = torch.zeros((len(pairs), 3), dtype=torch.int64, device="cuda")
    dpairs = torch.as_tensor(pairs, dtype=torch.int32, device="cuda")
    sums = g.count(dpairs, mask, per_edge=per)
    s, s2, lc = oracle_sums(rp, col, pairs)
    assert_sums_equal(sums, s, s2, ids)
    ref_pe = per_edge_reference(lc)
    got_pe = per.cpu().numpy()
    need_k = mask & (gs.GS_G7 | gs.GS_G8 | gs.GS_G9 | gs.GS_G11)
    need_q = mask & (gs.GS_G10 | gs.GS_G12)
    assert np.array_equal(got_pe[:, 0], ref_pe[:, 0])
    if need_k:
        assert np.array_equal(got_pe[:, 1], ref_pe[:, 1])
    if need_q:
        assert np.array_equal(got_pe[:, 2], ref_pe[:, 2])
    ref = oracle.estimate(s, s2, len(col) // 2, len(pairs))
    assert_estimates_close(gs.gs_estimate(sums), ref, ids)
    g.close()


# ------------------------------------------------------------------ small graphs

@pytest.mark.parametrize("gid", [3, 4, 7, 8, 9, 10, 11, 12])
def test_table1_graphlets_count_themselves(gid):
    n, edges = brute.GRAPHLET_EDGES[gid]
    rp, col = brute.csr_from_edges(n, edges)
    g = _graph(rp, col)
    res = gs.gs_estimate(g.count(None)).as_dict()
    want = brute.brute_counts(brute.adjacency(n, edges))
    for i in ALL:
        assert res[i]["exact"] == want[i], (gid, i)
    g.close()


def test_random_small_graphs_exact_against_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(25):
        n = int(rng.integers(5, 13))
        U = np.triu(rng.random((n, n)) < rng.uniform(0.2, 0.9), 1)
        A = (U | U.T).astype(np.int64)
        rp, col = brute.csr_from_adjacency(A)
        if len(col) == 0:
            continue
        g = _graph(rp, col)
        res = gs.gs_estimate(g.count(None)).as_dict()
        want = brute.brute_counts(A)
        for i in ALL:
            assert res[i]["exact"] == want[i], (trial, i)
        g.close()


@pytest.mark.parametrize("kind,args", [("complete", (40,)), ("cycle", (1000,)), ("star", (3000,)),
                                       ("bipartite", (50, 70)), ("path", (5000,))])
def test_closed_forms(kind, args):
    n, edges = brute.family_edges(kind, *args)
    rp, col = brute.csr_from_edges(n, edges) if n <= 200 else synth.from_pairs(
        n, np.array([e[0] for e in edges]), np.array([e[1] for e in edges]))
    g = _graph(rp, col)
    res = gs.gs_estimate(g.count(None)).as_dict()
    want = brute.closed_form(kind, *args)
    for i in ALL:
        assert res[i]["exact"] == want[i], (kind, i)
    g.close()


# ------------------------------------------------------------------ workloads

def test_er_2000_exact_and_explicit_sample():
    """Erdos-Renyi G(2000, 20000): exact counts (all edges) and a seeded 10%
    explicit edge list (shuffled, random orientation)."""
    rp, col = synth.er_2000()
    pairs_all = synth.upper_pairs(rp, col)
    _full_check(rp, col, pairs_all)
    sample = synth.explicit_sample(rp, col, 0.10, seed=2024)
    _full_check(rp, col, sample)
    g = _graph(rp, col)
    res = gs.gs_estimate(g.count(None)).as_dict()
    exact = oracle.exact_counts(rp, col)
    for i in ALL:
        assert res[i]["exact"] == exact[i]
    g.close()


@pytest.mark.parametrize("maker", [
    lambda: synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77),
    lambda: synth.rmat(13, 12, seed=5),
    lambda: synth.rgg(6000, 0.04, seed=8),
], ids=["chung_lu_20k", "rmat_13", "rgg_6k"])
@pytest.mark.parametrize("hub_budget", [0, NO_HUBS, 3 << 20], ids=["hubs", "no_hubs", "few_hubs"])
def test_medium_graphs_all_edges_and_samples(maker, hub_budget):
    rp, col = maker()
    g = _graph(rp, col, hub_budget_bytes=hub_budget)
    info = g.info
    g.close()
    if hub_budget == NO_HUBS:
        assert info["bitmap_hubs"] == 0 and info["table_hubs"] == 0
    _full_check(rp, col, synth.upper_pairs(rp, col), hub_budget=hub_budget)
    _full_check(rp, col, synth.explicit_sample(rp, col, 0.05, seed=1), hub_budget=hub_budget)


def test_hub_index_is_used_on_power_law_graphs():
    rp, col = synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77)
    g = _graph(rp, col)
    assert g.info["bitmap_hubs"] > 0 and g.info["table_hubs"] > 1
    assert g.info["matrix_hubs"] > 1
    assert g.info["mid_rows"] > 0 and 0 < g.info["big_hubs"] <= g.info["table_hubs"]
    assert g.info["dir_vertices"] > 0
    g.close()
    # a small budget still has directories (the highest degrees first); none at 1 byte
    few = _graph(rp, col, hub_budget_bytes=3 << 20)
    assert few.info["dir_vertices"] > 0
    few.close()
    none = _graph(rp, col, hub_budget_bytes=NO_HUBS)
    assert none.info["dir_vertices"] == 0
    none.close()


def test_mid_big_table_cut_by_budget():
    # a budget that leaves room for only part of the mid x big table: the
    # rows kept are the highest-degree mid vertices, the rest fall back to
    # searches, and the counts do not change
    rp, col = synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77)
    g = _graph(rp, col)
    full = g.info
    g.close()
    assert full["mid_rows"] > 0
    for budget in (1 << 20, 2 << 20, 3 << 20, 4 << 20, 6 << 20, 8 << 20, 12 << 20):
        g = _graph(rp, col, hub_budget_bytes=budget)
        info = g.info
        g.close()
        if 0 < info["mid_rows"] < full["mid_rows"]:
            break
    else:
        pytest.fail("no budget cut the mid x big table")
    _full_check(rp, col, synth.upper_pairs(rp, col), hub_budget=budget)
    _full_check(rp, col, synth.explicit_sample(rp, col, 0.1, seed=4), hub_budget=budget)


@pytest.mark.parametrize("mask", [gs.GS_G3, gs.GS_THREE_NODE, gs.GS_G7, gs.GS_G10,
                                  gs.GS_G8 | gs.GS_G12, gs.GS_G11, gs.GS_CONNECTED])
def test_masks_select_passes(mask):
    rp, col = synth.chung_lu(5000, 40000, 2.1, 600.0, seed=12)
    pairs = synth.explicit_sample(rp, col, 0.2, seed=3)
    ids = [g for g in ALL if mask & (1 << g)]
    _full_check(rp, col, pairs, mask=mask, ids=ids)


def test_sampler_matches_oracle_bit_exact():
    for rp, col in (synth.er_2000(), synth.chung_lu(50000, 400000, 2.1, 3000.0, seed=4)):
        g = _graph(rp, col)
        for frac, seed in ((0.01, 1), (0.1, 77), (0.5, 3), (1.0, 5), (0.0, 9)):
            got = g.sample(frac, seed).cpu().numpy()
            want = oracle.sample(rp, col, frac, seed)
            assert np.array_equal(got, want), (frac, seed)
        g.close()


def test_count_estimate_fused_matches_oracle():
    rp, col = synth.chung_lu(8000, 60000, 2.1, 900.0, seed=21)
    g = _graph(rp, col)
    res, k = g.count_estimate(0.1, seed=42)
    pairs = oracle.sample(rp, col, 0.1, 42)
    assert k == len(pairs)
    s, s2, _ = oracle_sums(rp, col, pairs)
    assert_estimates_close(res, oracle.estimate(s, s2, len(col) // 2, k), ALL)
    res1, k1 = g.count_estimate(1.0)
    exact = oracle.exact_counts(rp, col)
    got = res1.as_dict()
    for i in ALL:
        assert got[i]["exact"] == exact[i]
        assert got[i]["V"] == 0.0
    g.close()


# ------------------------------------------------------------------ edge cases

def test_empty_and_single_edge_samples():
    rp, col = synth.er(500, 3000, seed=1)
    g = _graph(rp, col)
    empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    s = g.count(empty)
    r = gs.gs_estimate(s)
    assert s.k == 0 and all(v == (0, 0) for v in s.sums().values())
    one = torch.as_tensor(synth.upper_pairs(rp, col)[:1], device="cuda")
    r = gs.gs_estimate(g.count(one)).as_dict()
    for i in ALL:
        assert r[i]["flags"] & gs.GS_F_VAR_UNDEFINED
    g.close()


def test_isolated_vertices_and_tiny_graph():
    rp, col = synth.from_pairs(50, np.array([3, 3, 4]), np.array([4, 5, 5]))
    g = _graph(rp, col)
    r = gs.gs_estimate(g.count(None)).as_dict()
    assert r[3]["exact"] == 1 and r[4]["exact"] == 0
    g.close()


def test_hub_heavy_star_of_cliques():
    """A hub joined to many small cliques: degree skew within one edge set."""
    edges = []
    hub = 0
    nxt = 1
    for c in range(300):
        size = 3 + c % 6
        members = list(range(nxt, nxt + size))
        nxt += size
        edges += list(itertools.combinations(members, 2))
        edges += [(hub, m) for m in members]
    a = np.array([e[0] for e in edges])
    b = np.array([e[1] for e in edges])
    rp, col = synth.from_pairs(nxt, a, b)
    _full_check(rp, col, synth.upper_pairs(rp, col))
    _full_check(rp, col, synth.upper_pairs(rp, col), hub_budget=NO_HUBS)


def test_invalid_inputs_are_rejected():
    rp, col = synth.er(300, 2000, seed=2)
    g = _graph(rp, col)
    pairs = synth.upper_pairs(rp, col)[:10].copy()
    bad = pairs.copy()
    # a non-edge
    nz = set(map(tuple, synth.upper_pairs(rp, col)))
    u = next(x for x in range(300) if (0, x) not in nz and x != 0)
    bad[3] = (0, u)
    with pytest.raises(gs.GraphletError) as ei:
        g.count(torch.as_tensor(bad, device="cuda"))
    assert ei.value.status == 6
    # out of range id
    bad = pairs.copy()
    bad[0] = (0, 10**6)
    with pytest.raises(gs.GraphletError) as ei:
        g.count(torch.as_tensor(bad, device="cuda"))
    assert ei.value.status == 6
    # duplicate edge (in either orientation)
    dup = np.concatenate([pairs, pairs[2:3, ::-1]])
    with pytest.raises(gs.GraphletError) as ei:
        g.count(torch.as_tensor(np.ascontiguousarray(dup), device="cuda"))
    assert ei.value.status == 7
    # bad mask
    with pytest.raises(gs.GraphletError):
        g.count(torch.as_tensor(pairs, device="cuda"), mask=1 << 5)
    # the handle still works afterwards
    s, s2, _ = oracle_sums(rp, col, pairs)
    assert_sums_equal(g.count(torch.as_tensor(pairs, device="cuda")), s, s2, ALL)
    g.close()


@pytest.mark.parametrize("defect", ["unsorted", "selfloop", "dup", "asym"])
def test_invalid_csr_is_rejected(defect):
    rp, col = synth.er(100, 400, seed=3)
    col = col.copy()
    rp = rp.copy()
    v = int(np.argmax(np.diff(rp)))
    s, e = rp[v], rp[v + 1]
    if defect == "unsorted":
        col[s], col[s + 1] = col[s + 1], col[s]
        code = 2
    elif defect == "selfloop":
        col[s] = v
        col[s:e] = np.sort(col[s:e])
        code = 3
    elif defect == "dup":
        col[s + 1] = col[s]
        code = 4
    else:
        present = set(col[s:e].tolist()) | {v}
        y = next(x for x in range(100) if x not in present)
        col[s] = y
        col[s:e] = np.sort(col[s:e])
        code = 5
    with pytest.raises(gs.GraphletError) as ei:
        gs.Graph.from_numpy(rp, col)
    assert ei.value.status == code


# ------------------------------------------------------------------ dense clique mode

def _core_periphery(n_core=420, p_core=0.9, n_per=4000, per_deg=8, seed=3):
    """A dense core (every core edge has T with hundreds of hub members) and
    a sparse periphery of low-degree vertices attached to the core, so T mixes
    vertices with and without hub-matrix slots."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n_core, 1)
    keep = rng.random(len(iu[0])) < p_core
    a = list(iu[0][keep])
    b = list(iu[1][keep])
    for i in range(n_per):
        for c in rng.choice(n_core, size=per_deg, replace=False):
            a.append(n_core + i)
            b.append(int(c))
    return synth.from_pairs(n_core + n_per, np.array(a), np.array(b))


def test_dense_clique_mode_closed_form():
    n, edges = brute.family_edges("complete", 300)
    rp, col = synth.from_pairs(n, np.array([e[0] for e in edges]), np.array([e[1] for e in edges]))
    g = _graph(rp, col)
    res = gs.gs_estimate(g.count(None)).as_dict()
    assert g.ws.stats()["dense_edges"] == g.m  # every edge's T is the other 298 vertices
    want = brute.closed_form("complete", 300)
    for i in ALL:
        assert res[i]["exact"] == want[i], i
    g.close()


def test_dense_clique_mode_mixed_t_against_oracle():
    rp, col = _core_periphery()
    sample = synth.explicit_sample(rp, col, 0.03, seed=9)
    g = _graph(rp, col)
    g.count(torch.as_tensor(sample, device="cuda"))
    st = g.ws.stats()
    assert 0 < st["dense_edges"] < len(sample)  # core edges dense, periphery edges not
    g.close()
    _full_check(rp, col, sample)
    _full_check(rp, col, sample, hub_budget=NO_HUBS)


@pytest.mark.parametrize("slots", [384, 0, 1 << 20])
def test_dense_slots_below_the_matrix_size(slots):
    """Only the first `slots` matrix slots take part in dense mode; the other
    matrix vertices of a dense edge's T scan their adjacency (rest mode) and
    still answer single tests from the matrix. 0 turns dense mode off; a
    count above the matrix size means every slot. (With 256 slots the cost
    model already prefers plain tests on this graph.)"""
    rp, col = _core_periphery()
    sample = synth.explicit_sample(rp, col, 0.03, seed=9)
    g = _graph(rp, col)
    assert g.info["matrix_hubs"] > 384  # the whole core has matrix slots
    g.ws.set_dense_slots(slots)
    g.count(torch.as_tensor(sample, device="cuda"))
    st = g.ws.stats()
    if slots:
        assert 0 < st["dense_edges"] < len(sample)
    else:
        assert st["dense_edges"] == 0
    g.close()
    _full_check(rp, col, sample, dense_slots=slots)


def test_dense_slots_complete_graph():
    n, edges = brute.family_edges("complete", 300)
    rp, col = synth.from_pairs(n, np.array([e[0] for e in edges]), np.array([e[1] for e in edges]))
    g = _graph(rp, col)
    g.ws.set_dense_slots(256)
    res = gs.gs_estimate(g.count(None)).as_dict()
    assert g.ws.stats()["dense_edges"] == g.m
    want = brute.closed_form("complete", 300)
    for i in ALL:
        assert res[i]["exact"] == want[i], i
    with pytest.raises(gs.GraphletError):
        g.ws.set_dense_slots(-1)
    g.close()


# ------------------------------------------------------------------ giant hubs

def test_giant_hub_pair_codegree_above_16_bits():
    """K_{2,70000}: the two hubs share 70,000 neighbours, more than a 16-bit
    co-degree entry holds, so c(a, b) must come from the 32-bit table of
    giant pairs; every sampled leaf edge (x, b) has w = a in S_x and
    q = c(a, b) - 1."""
    n = 70000
    leaves = np.arange(2, n + 2, dtype=np.int64)
    a = np.concatenate([np.zeros(n, dtype=np.int64), np.ones(n, dtype=np.int64)])
    b = np.concatenate([leaves, leaves])
    rp, col = synth.from_pairs(n + 2, a, b)
    g = _graph(rp, col)
    assert g.info["table_hubs"] == 2
    g.close()
    sample = synth.explicit_sample(rp, col, 0.002, seed=5)
    _full_check(rp, col, sample)
