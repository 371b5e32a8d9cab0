"""The oracle's per-edge local counts, run by a pool of spawned processes
(test infrastructure). The CSR is shared through memory-mapped .npy files;
every worker runs the unchanged single-threaded oracle on a chunk of the
edge list and the chunks are concatenated in order, so the result is the
oracle's own per-edge output. The pool is started with ``spawn`` so that it
never inherits a CUDA context."""
import multiprocessing as mp
import os
import sys
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

_CSR = None


def _init(rp_path, col_path):
    global _CSR
    sys.path.insert(0, ROOT)
    _CSR = (np.load(rp_path, mmap_mode="r"), np.load(col_path, mmap_mode="r"))


def _chunk(job):
    import oracle
    pairs, four = job
    rp, col = _CSR
    return oracle.local_counts(np.asarray(rp), np.asarray(col), pairs, four=four)


def _micro_chunk(job):
    import oracle
    pairs, p_e, seed = job
    rp, col = _CSR
    return oracle.micro(np.asarray(rp), np.asarray(col), pairs, p_e, seed)


class OraclePool:
    """with OraclePool(rp, col) as pool: lc = pool.local_counts(pairs)"""

    def __init__(self, rp, col, workers=None):
        self.workers = workers or os.cpu_count() or 1
        self.tmp = tempfile.mkdtemp(prefix="gs_oracle_pool_")
        self.rp_path = os.path.join(self.tmp, "rp.npy")
        self.col_path = os.path.join(self.tmp, "col.npy")
        np.save(self.rp_path, np.asarray(rp, dtype=np.int64))
        np.save(self.col_path, np.asarray(col, dtype=np.int32))
        self.pool = mp.get_context("spawn").Pool(self.workers, _init,
                                                 (self.rp_path, self.col_path))

    def local_counts(self, pairs, four=True, chunks_per_worker=8):
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        if len(pairs) == 0:
            return {x: np.zeros(0, dtype=np.int64) for x in ("t", "a", "b", "k", "q")}
        step = max(1, -(-len(pairs) // (self.workers * chunks_per_worker)))
        jobs = [(pairs[i:i + step], four) for i in range(0, len(pairs), step)]
        parts = self.pool.map(_chunk, jobs, chunksize=1)
        return {x: np.concatenate([p[x] for p in parts]) for x in ("t", "a", "b", "k", "q")}

    def micro(self, pairs, p_e=1.0, seed=0, chunks_per_worker=8):
        """oracle.micro over the pool (rows in input order)."""
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        if len(pairs) == 0:
            return np.zeros((0, 15)), np.zeros(0)
        step = max(1, -(-len(pairs) // (self.workers * chunks_per_worker)))
        jobs = [(pairs[i:i + step], p_e, seed) for i in range(0, len(pairs), step)]
        parts = self.pool.map(_micro_chunk, jobs, chunksize=1)
        return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))

    def close(self):
        self.pool.close()
        self.pool.join()
        for f in (self.rp_path, self.col_path):
            os.remove(f)
        os.rmdir(self.tmp)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
