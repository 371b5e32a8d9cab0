"""Disconnected graphlets (G5, G6, G13-G17) on the GPU: the folded sums,
estimates and exact counts against the oracle's reading of Sec. 2.3 and
against brute force."""
import math

import numpy as np
import pytest

import brute
import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402


def _close(a, b, tol=1e-12):
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return abs(a - b) <= tol * max(abs(a), abs(b), 1.0)


def _check(rp, col, pairs_np):
    g = gs.Graph.from_numpy(rp, col)
    pairs = torch.as_tensor(pairs_np, dtype=torch.int32, device="cuda")
    conn, disc = g.count_all(pairs)
    assert disc.k == len(pairs_np) and disc.m == len(col) // 2 and disc.n == len(rp) - 1
    got = gs.gs_estimate_disconnected(disc).as_dict()
    want = oracle.disconnected_estimate(rp, col, pairs_np)
    for gid in gs.DISCONNECTED:
        assert _close(got[gid]["X"], want[gid]["X"]), (gid, got[gid]["X"], want[gid]["X"])
        assert _close(got[gid]["V"], want[gid]["V"]), (gid, got[gid]["V"], want[gid]["V"])
        assert got[gid]["exact"] == want[gid]["exact"], gid
    g.close()
    return got


@pytest.mark.parametrize("maker", [
    lambda: synth.er_2000(),
    lambda: synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77),
    lambda: synth.rmat(12, 10, seed=3),
], ids=["er_2000", "chung_lu_20k", "rmat_12"])
def test_disconnected_estimates_match_oracle(maker):
    rp, col = maker()
    _check(rp, col, synth.upper_pairs(rp, col))                       # exact
    _check(rp, col, synth.explicit_sample(rp, col, 0.1, seed=2))     # estimate


def test_disconnected_exact_counts_match_brute_force_on_small_graphs():
    rng = np.random.default_rng(42)
    for _ in range(25):
        n = int(rng.integers(4, 13))
        A = np.triu((rng.random((n, n)) < rng.random()).astype(np.int64), 1)
        A = A + A.T
        if A.sum() == 0:
            continue
        rp, col = brute.csr_from_adjacency(A)
        got = _check(rp, col, synth.upper_pairs(rp, col))
        want = brute.brute_counts(A)
        for gid in gs.DISCONNECTED:
            assert got[gid]["exact"] == want[gid], (gid, got[gid]["exact"], want[gid])


def test_count_all_without_pairs_counts_every_edge():
    rp, col = synth.er(500, 4000, seed=9)
    g = gs.Graph.from_numpy(rp, col)
    conn, disc = g.count_all()
    assert disc.k == disc.m == g.m
    res = gs.gs_estimate_disconnected(disc).as_dict()
    n = len(rp) - 1
    three = sum(gs.gs_estimate(conn).as_dict()[i]["exact"] for i in (3, 4))
    assert three + res[5]["exact"] + res[6]["exact"] == math.comb(n, 3)
    g.close()


def test_disconnected_rejects_pairs_outside_the_graph():
    rp, col = synth.er(100, 300, seed=1)
    g = gs.Graph.from_numpy(rp, col)
    pairs = torch.tensor([[0, 5000]], dtype=torch.int32, device="cuda")
    per = torch.zeros((1, 3), dtype=torch.int64, device="cuda")
    with pytest.raises(gs.GraphletError):
        gs.gs_count_disconnected(g.handle, g.ws.handle, pairs, 1, per)
    g.close()


def test_per_edge_numerator_rows_match_the_oracle_and_sum_to_the_totals():
    rp, col = synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77)
    g = gs.Graph.from_numpy(rp, col)
    pairs_np = synth.explicit_sample(rp, col, 0.05, seed=6)
    pairs = torch.as_tensor(pairs_np, dtype=torch.int32, device="cuda")
    k = pairs.shape[0]
    per = torch.empty((k, 3), dtype=torch.int64, device="cuda")
    sums = g.count(pairs, gs.GS_CONNECTED, per_edge=per)
    rows = torch.empty((k, 8), dtype=torch.int64, device="cuda")
    gs.gs_per_edge_numerators(g.handle, g.ws.handle, pairs, k, per, rows)
    got = rows.cpu().numpy()
    _, _, want = oracle.numerators(oracle.local_counts(rp, col, pairs_np), per_edge=True)
    assert np.array_equal(got, want)
    tot = sums.sums()
    for i, gid in enumerate(gs.GRAPHLETS):
        assert int(got[:, i].astype(object).sum()) == tot[gid][0]
    g.close()
