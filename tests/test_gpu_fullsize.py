"""Parity at full workload sizes, in the launch configuration bench.py times.

The oracle cannot count every edge of these graphs, so the checks are:
  * the library's sampler output equals the oracle sampler's, bit for bit;
  * per-edge (t, k, q) of a few hundred sampled edges, recomputed one by one
    by the oracle, equal the library's per-edge output for the same edges;
  * exact counts at fraction 1 satisfy counting identities that hold at any
    size (degree sums and 3-path counts fix linear combinations of the
    induced counts).
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402


def _exact_sum(vals: np.ndarray) -> int:
    """Exact sum of non-negative int64 values as a Python int (large values
    are summed one by one, the rest in chunks that cannot overflow)."""
    big = vals > (1 << 40)
    total = sum(int(v) for v in vals[big])
    small = vals[~big]
    return total + sum(int(c.sum()) for c in np.array_split(small, max(1, len(small) >> 20)))


def _degree_identities(rp, col):
    d = np.diff(rp).astype(np.int64)
    src = np.repeat(np.arange(len(d), dtype=np.int64), d)
    up = src < col
    du = d[src[up]] - 1
    dv = d[col[up]] - 1
    wedges = _exact_sum(d * (d - 1) // 2)
    claws = _exact_sum(d * (d - 1) * (d - 2) // 6)
    paths = _exact_sum(du * dv)
    return wedges, claws, paths


def _per_edge_spot_check(g, rp, col, pairs_dev, mask, count, seed):
    k = pairs_dev.shape[0]
    per = torch.zeros((k, 3), dtype=torch.int64, device="cuda")
    g.count(pairs_dev, mask, per_edge=per)
    pe = per.cpu().numpy()
    pairs = pairs_dev.cpu().numpy()
    rng = np.random.default_rng(seed)
    idx = rng.choice(k, size=min(count, k), replace=False)
    lc = oracle.local_counts(rp, col, pairs[idx])
    assert np.array_equal(pe[idx, 0], lc["t"])
    if mask & (gs.GS_G7 | gs.GS_G8 | gs.GS_G9 | gs.GS_G11):
        assert np.array_equal(pe[idx, 1], lc["k"])
    if mask & (gs.GS_G10 | gs.GS_G12):
        assert np.array_equal(pe[idx, 2], lc["q"])


def test_chung_lu_1m_full_size():
    gs.build()
    rp, col = synth.chung_lu_1m()
    g = gs.Graph.from_numpy(rp, col)
    # sampler: bit-exact at 1%
    pairs = g.sample(0.01, 1)
    assert np.array_equal(pairs.cpu().numpy(), oracle.sample(rp, col, 0.01, 1))
    _per_edge_spot_check(g, rp, col, pairs, gs.GS_CONNECTED, 300, 3)
    # exact counts of every edge: identities at full size
    t0 = time.time()
    res = gs.gs_estimate(g.count(None, gs.GS_CONNECTED)).as_dict()
    print("exact connected counts, all edges:", round(time.time() - t0, 2), "s")
    c = {i: res[i]["exact"] for i in gs.GRAPHLETS}
    assert all(v is not None for v in c.values())
    wedges, claws, paths = _degree_identities(rp, col)
    assert wedges == c[4] + 3 * c[3]
    assert claws == c[11] + c[9] + 2 * c[8] + 4 * c[7]
    assert paths - 3 * c[3] == c[12] + 2 * c[9] + 4 * c[10] + 6 * c[8] + 12 * c[7]
    g.close()


def test_rmat_24_full_size():
    gs.build()
    t0 = time.time()
    rp, col = synth.rmat_24()
    print("rmat_24 generated:", len(rp) - 1, "vertices,", len(col) // 2, "edges,",
          round(time.time() - t0, 1), "s")
    g = gs.Graph.from_numpy(rp, col)
    g.ws.set_timing(True)
    # exact 3-node counts over all edges: identity sum C(d,2) = G4 + 3 G3
    res = gs.gs_estimate(g.count(None, gs.GS_THREE_NODE)).as_dict()
    print("exact 3-node:", g.ws.stats())
    wedges, _, _ = _degree_identities(rp, col)
    assert wedges == res[4]["exact"] + 3 * res[3]["exact"]
    # 4-node estimates at 0.1% and 1%: sampler bit-exact, per-edge spot check
    for frac, seed in ((0.001, 7), (0.01, 8)):
        pairs = g.sample(frac, seed)
        assert np.array_equal(pairs.cpu().numpy(), oracle.sample(rp, col, frac, seed))
        _per_edge_spot_check(g, rp, col, pairs, gs.GS_CONNECTED, 150, seed)
        print(f"4-node at {frac}:", g.ws.stats())
    g.close()
