"""Parity at full workload sizes, in the launch configuration bench.py times.

The oracle (run by a pool of spawned processes, one per host core) checks:
  * the library's sampler output equals the oracle sampler's, bit for bit;
  * on the 1M-vertex Chung-Lu graph, every edge of the 1% sample: per-edge
    (t, k, q) and the exact sums of N_i and N_i^2;
  * per-edge (t, k, q) of degree-stratified edge sets, chosen where the
    index answers most of the work: the edges with the largest smaller
    degree (hub-hub edges), the edges with the largest triangle sets (the
    word-parallel dense mode), edges between two co-degree-table vertices,
    edges with one end among the mid x big table's columns, edges whose
    smaller end has a bucket directory, and a uniform remainder; on the
    exact pass over every edge (Chung-Lu) and the exact 3-node pass over
    every edge (R-MAT), and on the 4-node R-MAT samples (a prefix of the
    0.1% sample plus its hub edges; hub and uniform edges of the 1% sample);
  * the batched path on the real 4096-graph generator, every 32nd graph
    against the oracle's exact counts.
Degree-sum identities are kept as smoke checks only: they hold for any
triangle, clique and cycle counts.
"""
import time

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

FOUR_K = gs.GS_G7 | gs.GS_G8 | gs.GS_G9 | gs.GS_G11
FOUR_Q = gs.GS_G10 | gs.GS_G12


def _exact_sum(vals: np.ndarray) -> int:
    """Exact sum of non-negative int64 values as a Python int."""
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
    return (_exact_sum(d * (d - 1) // 2), _exact_sum(d * (d - 1) * (d - 2) // 6),
            _exact_sum(du * dv))


def _stratified(rp, pairs, t=None, n_top=500, n_each=300, seed=0):
    """Indices into `pairs` of the strata described in the module doc."""
    rng = np.random.default_rng(seed)
    d = np.diff(rp)
    du, dv = d[pairs[:, 0]], d[pairs[:, 1]]
    lo, hi = np.minimum(du, dv), np.maximum(du, dv)
    order = np.argsort(-d, kind="stable")
    rank = np.empty(len(d), dtype=np.int64)
    rank[order] = np.arange(len(d))
    ru, rv = rank[pairs[:, 0]], rank[pairs[:, 1]]
    picks = [np.argsort(-lo, kind="stable")[:n_top]]
    if t is not None:
        picks.append(np.argsort(-t, kind="stable")[:n_each])

    def some(mask):
        idx = np.flatnonzero(mask)
        return rng.choice(idx, size=min(n_each, len(idx)), replace=False) if len(idx) else idx

    picks.append(some((ru < 65535) & (rv < 65535)))                   # table x table
    picks.append(some((np.minimum(ru, rv) < 4096) & (np.maximum(ru, rv) >= 65535)))  # big x rest
    picks.append(some((lo >= 16) & (lo <= 4096)))                      # directory-tested
    picks.append(some(hi >= 65536))                                    # a giant end
    picks.append(rng.choice(len(pairs), size=min(n_each, len(pairs)), replace=False))
    return np.unique(np.concatenate(picks))


def _check_rows(pe, lc, idx, mask):
    assert np.array_equal(pe[:, 0], lc["t"][idx] if idx is not None else lc["t"])
    sel = (lambda a: a[idx]) if idx is not None else (lambda a: a)
    if mask & FOUR_K:
        assert np.array_equal(pe[:, 1], sel(lc["k"]))
    if mask & FOUR_Q:
        assert np.array_equal(pe[:, 2], sel(lc["q"]))


def _count_per_edge(g, pairs_dev, mask):
    k = g.m if pairs_dev is None else pairs_dev.shape[0]
    per = torch.zeros((k, 3), dtype=torch.int64, device="cuda")
    sums = g.count(pairs_dev, mask, per_edge=per)
    return sums, per


def test_chung_lu_1m_full_size():
    gs.build()
    rp, col = synth.chung_lu_1m()
    g = gs.Graph.from_numpy(rp, col)
    with OraclePool(rp, col) as pool:
        # 1%: every sampled edge, per edge and the exact sums
        pairs = g.sample(0.01, 1)
        pnp = pairs.cpu().numpy()
        assert np.array_equal(pnp, oracle.sample(rp, col, 0.01, 1))
        sums, per = _count_per_edge(g, pairs, gs.GS_CONNECTED)
        t0 = time.time()
        lc = pool.local_counts(pnp)
        print(f"oracle over the whole 1% sample ({len(pnp)} edges): {time.time() - t0:.1f} s")
        _check_rows(per.cpu().numpy(), lc, None, gs.GS_CONNECTED)
        s, s2 = oracle.numerators(lc)
        assert all(sums.sums()[gid] == (s[gid], s2[gid]) for gid in gs.GRAPHLETS)
        # 5% and 10%: sampler bit-exact, stratified per-edge rows
        for frac, seed in ((0.05, 2), (0.10, 3)):
            pairs = g.sample(frac, seed)
            pnp = pairs.cpu().numpy()
            assert np.array_equal(pnp, oracle.sample(rp, col, frac, seed))
            _, per = _count_per_edge(g, pairs, gs.GS_CONNECTED)
            pe = per.cpu().numpy()
            idx = _stratified(rp, pnp, t=pe[:, 0], n_top=200, n_each=150, seed=seed)
            _check_rows(pe[idx], pool.local_counts(pnp[idx]), None, gs.GS_CONNECTED)
        # exact pass over every edge (canonical order): stratified rows
        sums, per = _count_per_edge(g, None, gs.GS_CONNECTED)
        assert g.ws.stats()["dense_edges"] > 0  # the word-parallel mode was taken
        allp = synth.upper_pairs(rp, col)
        t_all = per[:, 0].cpu().numpy()
        idx = _stratified(rp, allp, t=t_all, seed=7)
        pe = per[torch.as_tensor(idx, device="cuda")].cpu().numpy()
        t0 = time.time()
        _check_rows(pe, pool.local_counts(allp[idx]), None, gs.GS_CONNECTED)
        print(f"exact pass: {len(idx)} stratified edges checked in {time.time() - t0:.1f} s")
    # smoke: the degree identities of the exact counts
    res = gs.gs_estimate(sums).as_dict()
    c = {i: res[i]["exact"] for i in gs.GRAPHLETS}
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
    with OraclePool(rp, col) as pool:
        # exact 3-node counts over every edge: stratified per-edge t
        sums, per = _count_per_edge(g, None, gs.GS_THREE_NODE)
        print("exact 3-node:", g.ws.stats())
        allp = synth.upper_pairs(rp, col)
        idx = _stratified(rp, allp, n_top=1000, n_each=500, seed=11)
        pe = per[torch.as_tensor(idx, device="cuda")].cpu().numpy()
        del per
        lc = pool.local_counts(allp[idx], four=False)
        assert np.array_equal(pe[:, 0], lc["t"])
        res = gs.gs_estimate(sums).as_dict()
        wedges, _, _ = _degree_identities(rp, col)
        assert wedges == res[4]["exact"] + 3 * res[3]["exact"]  # smoke only
        # 4-node samples: sampler bit-exact; a prefix plus the hub edges of
        # the 0.1% sample, hub and uniform edges of the 1% sample
        for frac, seed, prefix, n_top, n_each in ((0.001, 7, 6000, 96, 100),
                                                  (0.01, 8, 0, 64, 100)):
            pairs = g.sample(frac, seed)
            pnp = pairs.cpu().numpy()
            assert np.array_equal(pnp, oracle.sample(rp, col, frac, seed))
            _, per = _count_per_edge(g, pairs, gs.GS_CONNECTED)
            pe = per.cpu().numpy()
            idx = _stratified(rp, pnp, t=pe[:, 0], n_top=n_top, n_each=n_each, seed=seed)
            idx = np.unique(np.concatenate([idx, np.arange(min(prefix, len(pnp)))]))
            t0 = time.time()
            lc = pool.local_counts(pnp[idx])
            _check_rows(pe[idx], lc, None, gs.GS_CONNECTED)
            print(f"4-node at {frac}: {len(idx)} edges checked in {time.time() - t0:.1f} s;",
                  g.ws.stats())
    g.close()


def test_batched_path_on_the_4096_graph_generator():
    """The batched configuration's own generator (n ~ U{50..5000}, mean degree
    ~ U[4, 40], ER / Chung-Lu 2.3 / 2-D RGG): exact counts of every 32nd
    graph equal the oracle's."""
    gs.build()
    graphs = synth.batch_4096()
    b = gs.Batch.from_graphs(graphs, autotune=False)
    exact = b.exact()
    for i in range(0, len(graphs), 32):
        rp, col = graphs[i]
        want = oracle.exact_counts(rp, col)
        assert exact[i] == want, (i, exact[i], want)
    b.close()
