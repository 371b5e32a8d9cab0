"""Seeded synthetic inputs shared by the CPU oracle, the tests and the bench.

This module holds no arithmetic of the graphlet method: it only generates
simple undirected graphs (int64 row offsets + int32 sorted adjacency, both
orientations stored) and explicit edge lists drawn with its own RNG.  Every
output is a pure function of its arguments and seed.

Workload recipes (stand-ins for the network-repository graphs the paper
evaluates on, which are not available here):

* ``er_2000``      Erdos-Renyi G(n=2000, m=20000), exactly m distinct pairs.
* ``chung_lu_1m``  Chung-Lu, n=1,000,000, m~20M, degree exponent 2.1,
                   expected degree capped at 50,000.
* ``rmat_24``      R-MAT scale 24, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05),
                   symmetrised, deduplicated, self-loops removed.
* ``batch_4096``   4096 small graphs, n ~ U{50..5000}, average degree
                   ~ U[4,40], model uniform over {ER, Chung-Lu 2.3, 2-D RGG}.
Vertex labels are randomly permuted after generation.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
BASE_SEED = 0x170101772


def build(force: bool = False) -> str:
    """Compiles gen.c into _synth.so (OpenMP if the compiler has it)."""
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", src, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


@functools.lru_cache(maxsize=1)
def _lib() -> ctypes.CDLL:
    lib = ctypes.CDLL(build())
    P, I64, U64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
    lib.synth_rmat.argtypes = [I, I64, D, D, D, U64, I]
    lib.synth_chung_lu.argtypes = [I64, I64, D, D, D, U64, I]
    lib.synth_er.argtypes = [I64, I64, U64, I]
    lib.synth_rgg.argtypes = [I64, D, U64, I]
    lib.synth_from_pairs.argtypes = [I64, I64, P, P]
    for f in ("synth_rmat", "synth_chung_lu", "synth_er", "synth_rgg", "synth_from_pairs"):
        getattr(lib, f).restype = P
    lib.synth_csr_n.argtypes = [P]
    lib.synth_csr_n.restype = I64
    lib.synth_csr_nnz.argtypes = [P]
    lib.synth_csr_nnz.restype = I64
    lib.synth_csr_copy.argtypes = [P, P, P]
    lib.synth_csr_free.argtypes = [P]
    lib.synth_threads.restype = I
    return lib


def _take(h) -> tuple[np.ndarray, np.ndarray]:
    if not h:
        raise MemoryError("synthetic graph generation failed (allocation or bad arguments)")
    lib = _lib()
    n, nnz = lib.synth_csr_n(h), lib.synth_csr_nnz(h)
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(nnz, 1), dtype=np.int32)[:nnz]
    lib.synth_csr_copy(h, row_ptr.ctypes.data, col.ctypes.data if nnz else None)
    lib.synth_csr_free(h)
    return row_ptr, col


def from_pairs(n: int, a, b) -> tuple[np.ndarray, np.ndarray]:
    """Simple undirected CSR from unordered pairs (loops and repeats dropped)."""
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int32)
    return _take(_lib().synth_from_pairs(n, len(a), a.ctypes.data, b.ctypes.data))


def er(n: int, m: int, seed: int, permute: bool = True):
    return _take(_lib().synth_er(n, m, seed, int(permute)))


def rgg(n: int, radius: float, seed: int, permute: bool = True):
    return _take(_lib().synth_rgg(n, radius, seed, int(permute)))


def rmat(scale: int, edge_factor: int, seed: int, abc=(0.57, 0.19, 0.19), permute: bool = True):
    e = edge_factor << scale
    return _take(_lib().synth_rmat(scale, e, abc[0], abc[1], abc[2], seed, int(permute)))


def chung_lu(n: int, m: int, gamma: float, cap: float, seed: int, permute: bool = True):
    """Chung-Lu graph with about m distinct edges: draws are topped up until
    the deduplicated edge count reaches m (the draw stream is counter-based,
    so a longer run extends a shorter one)."""
    draws = m
    for _ in range(6):
        row_ptr, col = _take(_lib().synth_chung_lu(n, draws, gamma, cap, 2.0 * m, seed, int(permute)))
        got = len(col) // 2
        if got >= m * 0.999:
            return row_ptr, col
        draws = int(draws + (m - got) * (draws / max(got, 1)) * 1.02) + 16
    return row_ptr, col


def degrees(row_ptr: np.ndarray) -> np.ndarray:
    return np.diff(row_ptr)


def upper_pairs(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """All edges (u < v) in row-major CSR order, as an int32 [M, 2] array."""
    n = len(row_ptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(row_ptr))
    keep = src < col
    return np.stack([src[keep], col[keep]], axis=1)


def explicit_sample(row_ptr, col, fraction: float, seed: int, shuffle: bool = True) -> np.ndarray:
    """An explicit sampled-edge list: each edge kept independently with
    probability `fraction` (this module's own RNG, not the method's sampler),
    then shuffled and with random orientation, as a caller might pass it."""
    pairs = upper_pairs(row_ptr, col)
    rng = np.random.default_rng(seed)
    keep = rng.random(len(pairs)) < fraction
    out = pairs[keep].copy()
    if shuffle:
        out = out[rng.permutation(len(out))]
        flip = rng.random(len(out)) < 0.5
        out[flip] = out[flip][:, ::-1]
    return np.ascontiguousarray(out, dtype=np.int32)


# ------------------------------------------------------------ named workloads

@functools.lru_cache(maxsize=4)
def er_2000(seed: int = BASE_SEED + 0):
    return er(2000, 20000, seed)


@functools.lru_cache(maxsize=2)
def chung_lu_1m(seed: int = BASE_SEED + 1):
    return chung_lu(1_000_000, 20_000_000, 2.1, 50_000.0, seed)


@functools.lru_cache(maxsize=1)
def rmat_24(seed: int = BASE_SEED + 2):
    return rmat(24, 16, seed)


def chung_lu_100k(seed: int):
    return chung_lu(100_000, 2_000_000, 2.1, 50_000.0, seed)


def small_graph(kind: int, n: int, avg_deg: float, seed: int):
    """One member of the batched workload: kind 0 = ER, 1 = Chung-Lu with
    exponent 2.3 (expected degree capped at n/2), 2 = 2-D RGG with radius
    sqrt(avg_deg / (pi n))."""
    m = int(round(n * avg_deg / 2))
    m = min(m, n * (n - 1) // 2)
    if kind == 0:
        return er(n, m, seed)
    if kind == 1:
        return chung_lu(n, m, 2.3, max(n / 2.0, 2.0), seed)
    return rgg(n, float(np.sqrt(avg_deg / (np.pi * n))), seed)


def batch_specs(count: int, seed: int = BASE_SEED + 3, n_range=(50, 5000), deg_range=(4.0, 40.0)):
    """(kind, n, avg_deg, seed) for each graph of a batched workload."""
    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, 3, size=count)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    degs = rng.uniform(deg_range[0], deg_range[1], size=count)
    seeds = rng.integers(1, 2**62, size=count)
    return [(int(k), int(n), float(d), int(s)) for k, n, d, s in zip(kinds, ns, degs, seeds)]


def pack(graphs):
    """Packs a list of (row_ptr, col) into one CSR with per-graph offsets.

    Returns (vtx_off int64[G+1], nnz_off int64[G+1], row_ptr int64[sumN+1]
    with global offsets into col, col int32[sumNNZ] with LOCAL vertex ids)."""
    g = len(graphs)
    vtx_off = np.zeros(g + 1, dtype=np.int64)
    nnz_off = np.zeros(g + 1, dtype=np.int64)
    for i, (rp, c) in enumerate(graphs):
        vtx_off[i + 1] = vtx_off[i] + len(rp) - 1
        nnz_off[i + 1] = nnz_off[i] + len(c)
    row_ptr = np.empty(vtx_off[-1] + 1, dtype=np.int64)
    col = np.empty(nnz_off[-1], dtype=np.int32)
    for i, (rp, c) in enumerate(graphs):
        row_ptr[vtx_off[i]:vtx_off[i + 1]] = rp[:-1] + nnz_off[i]
        col[nnz_off[i]:nnz_off[i + 1]] = c
    row_ptr[-1] = nnz_off[-1]
    return vtx_off, nnz_off, row_ptr, col


def batch_4096(count: int = 4096, seed: int = BASE_SEED + 3):
    return [small_graph(*spec) for spec in batch_specs(count, seed)]
