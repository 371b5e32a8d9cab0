"""Batched path: many small graphs counted exactly in one CUDA-graph launch,
checked graph by graph against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402


def _oracle_exact(rp, col):
    if len(col) == 0:
        return {g: 0 for g in gs.GRAPHLETS}
    return oracle.exact_counts(rp, col)


def _small_batch(count, seed, n_range=(50, 400), deg_range=(3.0, 20.0)):
    specs = synth.batch_specs(count, seed=seed, n_range=n_range, deg_range=deg_range)
    graphs = [synth.small_graph(*sp) for sp in specs]
    # edge cases: an edgeless graph, a single vertex, a 4-clique
    graphs.insert(3, synth.from_pairs(5, np.array([], dtype=np.int32), np.array([], dtype=np.int32)))
    graphs.insert(7, synth.from_pairs(1, np.array([], dtype=np.int32), np.array([], dtype=np.int32)))
    graphs.append(synth.from_pairs(4, np.array([0, 0, 0, 1, 1, 2]), np.array([1, 2, 3, 2, 3, 3])))
    return graphs


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_oracle_per_graph(autotune):
    gs.build()
    graphs = _small_batch(40, seed=11)
    b = gs.Batch.from_graphs(graphs, autotune=autotune)
    info = b.info()
    assert info["num_graphs"] == len(graphs)
    if autotune:
        assert info["candidates"] == 24 and info["best_ms"] <= info["worst_ms"]
    got = b.exact()
    for i, (rp, col) in enumerate(graphs):
        want = _oracle_exact(rp, col)
        for gid in gs.GRAPHLETS:
            assert got[i][gid] == want[gid], (i, gid, got[i][gid], want[gid])
    # the captured graph replays to the same sums
    again = b.count()
    first = b.count()
    for x, y in zip(again, first):
        assert x.sums() == y.sums()
    b.close()


def test_batch_sums_equal_single_graph_counts():
    gs.build()
    graphs = _small_batch(12, seed=5, n_range=(200, 1500), deg_range=(5.0, 30.0))
    b = gs.Batch.from_graphs(graphs, autotune=False)
    sums = b.count()
    for i, (rp, col) in enumerate(graphs):
        if len(col) == 0:
            assert sums[i].k == 0
            continue
        g = gs.Graph.from_numpy(rp, col)
        single = g.count(None, gs.GS_CONNECTED)
        assert sums[i].sums() == single.sums(), i
        assert sums[i].k == single.k == g.m
        g.close()
    b.close()


def test_batch_rejects_bad_local_ids():
    gs.build()
    graphs = [synth.er(30, 60, seed=1), synth.er(20, 40, seed=2)]
    vtx_off = np.array([0, 30, 50], dtype=np.int64)
    row_ptr = np.concatenate([graphs[0][0][:-1], graphs[1][0] + len(graphs[0][1])])
    col = np.concatenate([graphs[0][1], graphs[1][1]]).astype(np.int32)
    col[-1] = 25  # id 25 does not exist in the 20-vertex graph
    t = lambda a, dt: torch.as_tensor(a, dtype=dt, device="cuda")  # noqa: E731
    with pytest.raises(gs.GraphletError):
        gs.gs_batch_create(t(vtx_off, torch.int64), t(row_ptr, torch.int64), t(col, torch.int32))
