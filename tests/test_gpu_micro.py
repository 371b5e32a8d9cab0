"""Algorithm 7 (micro-level estimation) on the GPU against the oracle.

At p_e = 1 every statistic is an exact integer and the rows must equal the
oracle's bit for bit (x6 and x17 are rounded the same way on both sides);
4-clique and 4-cycle columns must also equal gs_count's per-edge k and q.
Below p_e = 1 both sides draw the same probe windows (seeded SplitMix64
offsets); the weighted sums differ only by rounding (fixed point on the
GPU, compensated FP64 sums in the oracle), so they agree within 1e-12 of
the magnitude of the terms involved. The column maxima and their first
edges (the extremal statistics of Sec. 7) must equal numpy's over the
oracle's rows."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle_pool import OraclePool

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402

REL = 1e-12
COL = {i: j for j, i in enumerate(gs.MICRO)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    yield


def _run(g, pairs_np, p_e, seed):
    pairs = torch.as_tensor(np.ascontiguousarray(pairs_np), device="cuda")
    out = torch.full((len(pairs_np), 15), float("nan"), dtype=torch.float64, device="cuda")
    mx, arg = gs.gs_micro(g.handle, g.ws.handle, pairs, len(pairs_np), p_e, seed, out)
    return out.cpu().numpy(), np.array(mx), np.array(arg)


def _first_argmax(x):
    return np.array([int(np.flatnonzero(x[:, j] == x[:, j].max())[0]) for j in range(x.shape[1])])


def _assert_close(got, want, om):
    """Sampled columns within REL of the terms they are made of."""
    samp = np.abs(want[:, [COL[7], COL[9], COL[10]]]).sum(1) + np.abs(om)
    for i in gs.MICRO:
        j = COL[i]
        scale = np.abs(want[:, j]) + samp + 1.0
        bad = np.abs(got[:, j] - want[:, j]) > REL * scale
        assert not bad.any(), (i, np.flatnonzero(bad)[:5], got[bad, j][:3], want[bad, j][:3])


GRAPHS = {
    "er_2000": lambda: synth.er_2000(),
    "chung_lu_20k": lambda: synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77),
    "rmat_13": lambda: synth.rmat(13, 12, seed=5),
    "rgg_6k": lambda: synth.rgg(6000, 0.025, seed=3),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_exact_micro_rows_equal_the_oracle_bit_for_bit(name):
    rp, col = GRAPHS[name]()
    g = gs.Graph.from_numpy(rp, col)
    pairs = synth.explicit_sample(rp, col, 0.2, seed=3)
    got, mx, arg = _run(g, pairs, 1.0, 9)
    assert g.ws.stats()["micro_probes"] > 0
    want, om = oracle.micro(rp, col, pairs, 1.0, 9)
    assert np.array_equal(got, want)
    # 4-cliques and 4-cycles per edge equal gs_count's
    per = torch.zeros((len(pairs), 3), dtype=torch.int64, device="cuda")
    g.count(torch.as_tensor(pairs, device="cuda"), gs.GS_CONNECTED, per_edge=per)
    pe = per.cpu().numpy()
    assert np.array_equal(got[:, COL[3]], pe[:, 0])
    assert np.array_equal(got[:, COL[7]], pe[:, 1])
    assert np.array_equal(got[:, COL[10]], pe[:, 2])
    assert np.array_equal(mx, want.max(0))
    assert np.array_equal(arg, _first_argmax(want))
    g.close()


@pytest.mark.parametrize("name", ["chung_lu_20k", "rmat_13"])
@pytest.mark.parametrize("p_e,seed", [(0.3, 4), (0.05, 5), (0.5, 2**63 + 11)])
def test_sampled_micro_rows_match_the_oracle(name, p_e, seed):
    rp, col = GRAPHS[name]()
    g = gs.Graph.from_numpy(rp, col)
    pairs = synth.explicit_sample(rp, col, 0.1, seed=6)
    got, mx, arg = _run(g, pairs, p_e, seed)
    want, om = oracle.micro(rp, col, pairs, p_e, seed)
    _assert_close(got, want, om)
    exact, _ = oracle.micro(rp, col, pairs, 1.0, 0)
    assert not np.array_equal(want[:, COL[7]], exact[:, COL[7]])  # probes were sampled
    # deterministic for a seed
    again, _, _ = _run(g, pairs, p_e, seed)
    assert np.array_equal(got, again)
    g.close()


def test_dense_graph_and_hub_edges():
    """K_200 plus a sparse periphery: every probe of a clique vertex lands in
    the hub-pair matrix or the adjacency blocks."""
    import itertools
    a, b = zip(*itertools.combinations(range(200), 2))
    rng = np.random.default_rng(3)
    extra = rng.integers(0, 3000, size=(6000, 2))
    extra = extra[extra[:, 0] != extra[:, 1]]
    a = np.concatenate([np.array(a), extra[:, 0]])
    b = np.concatenate([np.array(b), extra[:, 1]])
    rp, col = synth.from_pairs(3000, a, b)
    g = gs.Graph.from_numpy(rp, col)
    pairs = synth.upper_pairs(rp, col)
    got, mx, arg = _run(g, pairs, 1.0, 1)
    want, om = oracle.micro(rp, col, pairs, 1.0, 1)
    assert np.array_equal(got, want)
    # an edge of K_200 lies in at least C(198, 2) 4-cliques (periphery
    # vertices adjacent to three clique vertices add a few)
    assert mx[COL[7]] >= math.comb(198, 2)
    got, _, _ = _run(g, pairs, 0.2, 8)
    want, om = oracle.micro(rp, col, pairs, 0.2, 8)
    _assert_close(got, want, om)
    g.close()


def test_empty_and_invalid_samples():
    rp, col = synth.er(300, 2000, seed=2)
    g = gs.Graph.from_numpy(rp, col)
    empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros((0, 15), dtype=torch.float64, device="cuda")
    mx, arg = gs.gs_micro(g.handle, g.ws.handle, empty, 0, 0.5, 1, out)
    assert all(math.isnan(v) for v in mx) and all(i == -1 for i in arg)
    pairs = synth.upper_pairs(rp, col)[:10].copy()
    nz = set(map(tuple, synth.upper_pairs(rp, col)))
    bad = pairs.copy()
    bad[4] = next((0, y) for y in range(1, 300) if (0, y) not in nz)
    with pytest.raises(gs.GraphletError) as ei:
        _run(g, bad, 1.0, 0)
    assert ei.value.status == 6
    dup = np.concatenate([pairs, pairs[1:2, ::-1]])
    with pytest.raises(gs.GraphletError) as ei:
        _run(g, dup, 1.0, 0)
    assert ei.value.status == 7
    for p_e in (0.0, 1.5, float("nan")):
        with pytest.raises(gs.GraphletError) as ei:
            _run(g, pairs, p_e, 0)
        assert ei.value.status == 1
    got, _, _ = _run(g, pairs, 1.0, 0)  # still usable
    assert np.array_equal(got, oracle.micro(rp, col, pairs, 1.0, 0)[0])
    g.close()


def test_micro_on_the_1m_vertex_power_law_graph():
    """Chung-Lu 1M, the bench's graph and index: hub edges and uniform edges
    of a 1% sample at p_e = 0.01 and 1."""
    rp, col = synth.chung_lu_1m()
    g = gs.Graph.from_numpy(rp, col)
    pairs = g.sample(0.01, 1).cpu().numpy()
    d = np.diff(rp)
    lo = np.minimum(d[pairs[:, 0]], d[pairs[:, 1]])
    rng = np.random.default_rng(4)
    idx = np.unique(np.concatenate([np.argsort(-lo, kind="stable")[:40],
                                    rng.choice(len(pairs), 300, replace=False)]))
    sel = pairs[idx]
    with OraclePool(rp, col) as pool:
        for p_e, seed in ((0.01, 3), (1.0, 0)):
            got, mx, arg = _run(g, sel, p_e, seed)
            want, om = pool.micro(sel, p_e, seed)
            if p_e == 1.0:
                assert np.array_equal(got, want)
            else:
                _assert_close(got, want, om)
    g.close()
