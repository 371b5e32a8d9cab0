"""A sample sharded over two CUDA streams (two host threads, two
workspaces, counting at the same time on one GPU) and merged with
gs_sums_merge gives the unsharded sums bit for bit: the single-GPU
stand-in for the multi-GPU exchange, whose only step is this sum."""
import threading

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402


@pytest.mark.parametrize("mask", [gs.GS_THREE_NODE, gs.GS_CONNECTED])
def test_two_stream_shards_merge_to_the_unsharded_sums(mask):
    gs.build()
    rp, col = synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77)
    g = gs.Graph.from_numpy(rp, col)
    pairs = torch.as_tensor(synth.explicit_sample(rp, col, 0.2, seed=11), device="cuda")
    whole = g.count(pairs, mask)
    cut = pairs.shape[0] // 3  # uneven shards
    shards = [pairs[:cut].contiguous(), pairs[cut:].contiguous()]
    wss = [gs.Workspace(), gs.Workspace()]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    out, errs = [None, None], []

    def run(i):
        try:
            with torch.cuda.stream(streams[i]):
                out[i] = gs.gs_count(g.handle, wss[i].handle, shards[i], shards[i].shape[0], mask,
                                     stream=streams[i])
        except Exception as e:  # surfaced below
            errs.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs, errs
    merged = gs.gs_sums_merge(out[0], out[1])
    assert merged.k == whole.k == pairs.shape[0]
    assert merged.sums() == whole.sums()
    a, b = gs.gs_estimate(merged).as_dict(), gs.gs_estimate(whole).as_dict()
    for gid in a:
        assert np.isnan(a[gid]["X"]) == np.isnan(b[gid]["X"])
        assert a[gid]["X"] == b[gid]["X"] or (np.isnan(a[gid]["X"]) and np.isnan(b[gid]["X"]))
    for w in wss:
        w.close()
    g.close()
