"""The multi-GPU exchange, exercised on CPU: the sampled edge list is split
across world_size-2 gloo ranks, each rank folds its shard (here with the CPU
oracle standing in for its GPU), the per-rank sums are gathered and merged
exactly with gs_sums_merge, and the estimate equals the unsharded one."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import paper_1701_01772_gb300 as gs
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rp, col = synth.chung_lu(3000, 20000, 2.1, 400.0, seed=5)
    m = len(col) // 2
    pairs = oracle.sample(rp, col, 0.2, 13)
    shard = pairs[rank::world]  # disjoint shards of the same sample
    lc = oracle.local_counts(rp, col, shard)
    s, s2 = oracle.numerators(lc)
    mine = (len(shard), s, s2)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        acc = None
        for k, si, sq in gathered:
            part = gs.sums_from_ints(k, m, gs.GS_CONNECTED, si, sq)
            acc = part if acc is None else gs.gs_sums_merge(acc, part)
        merged = gs.gs_estimate(acc).as_dict()
        lc_all = oracle.local_counts(rp, col, pairs)
        s_all, s2_all = oracle.numerators(lc_all)
        whole = oracle.estimate(s_all, s2_all, m, len(pairs))
        ok = acc.k == len(pairs) and all(acc.sums()[g] == (s_all[g], s2_all[g])
                                         for g in gs.GRAPHLETS)
        for g in gs.GRAPHLETS:
            ok = ok and abs(merged[g]["X"] - whole[g]["X"]) <= 1e-12 * abs(whole[g]["X"])
        with open(out_path, "w") as f:
            f.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_sums_merge_exactly_over_two_gloo_ranks(tmp_path):
    import paper_1701_01772_gb300 as gs
    gs.build()
    out = tmp_path / "result.txt"
    mp.start_processes(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True,
                       start_method="spawn")
    assert out.read_text() == "ok"


def test_merge_rejects_mismatched_sums():
    import paper_1701_01772_gb300 as gs
    gs.build()
    a = gs.sums_from_ints(10, 100, gs.GS_CONNECTED, {}, {})
    b = gs.sums_from_ints(10, 99, gs.GS_CONNECTED, {}, {})
    with pytest.raises(gs.GraphletError):
        gs.gs_sums_merge(a, b)
    c = gs.sums_from_ints(95, 100, gs.GS_CONNECTED, {}, {})
    with pytest.raises(gs.GraphletError):
        gs.gs_sums_merge(a, c)
