"""Python binding of libgraphlet (C ABI in ``include/graphlet.h``).

Argument marshalling only: every step of the estimator runs in the CUDA
library. Device memory is passed as CUDA ``torch.Tensor`` objects, streams as
``torch.cuda.Stream`` (or None for the current stream). Function names match
the C entry points; ``Graph`` / ``Workspace`` are small owners of the opaque
handles.

If the compiled library is missing the import still succeeds (so that the
package can be built), but every call raises ``RuntimeError``: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

from .build import OUT as _LIB_PATH, build  # noqa: F401

GRAPHLETS = (3, 4, 7, 8, 9, 10, 11, 12)
DENOM = (3, 2, 6, 1, 2, 4, 6, 1)

GS_G3, GS_G4, GS_G7, GS_G8 = 1 << 3, 1 << 4, 1 << 7, 1 << 8
GS_G9, GS_G10, GS_G11, GS_G12 = 1 << 9, 1 << 10, 1 << 11, 1 << 12
GS_THREE_NODE = GS_G3 | GS_G4
GS_CONNECTED = GS_G3 | GS_G4 | GS_G7 | GS_G8 | GS_G9 | GS_G10 | GS_G11 | GS_G12
GS_VALIDATE = 1
GS_F_COMPUTED, GS_F_EXACT, GS_F_VAR_UNDEFINED, GS_F_OVERFLOW = 1, 2, 4, 8
GS_F_VAR_OVERFLOW = 16
# disconnected graphlets (gs_count_disconnected / gs_estimate_disconnected)
DISCONNECTED = (5, 6, 13, 14, 15, 16, 17)
DISC_DENOM = (1, 6, 6, 2, 2, 1, 12)

STATUS = {0: "GS_OK", 1: "GS_EINVAL", 2: "GS_ENOTSORTED", 3: "GS_ESELFLOOP", 4: "GS_EDUP",
          5: "GS_EASYM", 6: "GS_EEDGE", 7: "GS_EDUPSAMPLE", 8: "GS_EOVERFLOW", 9: "GS_ENOMEM",
          10: "GS_EBUDGET", 11: "GS_ETIMEOUT", 12: "GS_ECUDA", 13: "GS_ECAPACITY",
          14: "GS_ECANCELLED"}


class GraphletError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class GsSums(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("m", ctypes.c_int64), ("mask", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("sum", (ctypes.c_uint64 * 2) * 8),
                ("sumsq", (ctypes.c_uint64 * 2) * 8)]

    def sums(self) -> dict:
        """{graphlet: (sum N_i, sum N_i^2)} as Python ints."""
        out = {}
        for i, g in enumerate(GRAPHLETS):
            s = (int(self.sum[i][1]) << 64) | int(self.sum[i][0])
            if s >> 127:
                s -= 1 << 128
            s2 = (int(self.sumsq[i][1]) << 64) | int(self.sumsq[i][0])
            out[g] = (s, s2)
        return out


class GsSumsDisc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("overflow", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("sum", (ctypes.c_uint64 * 2) * 7), ("sumsq", (ctypes.c_uint64 * 2) * 7)]

    def sums(self) -> dict:
        """{graphlet: (sum N_i, sum N_i^2)} as Python ints (order of DISCONNECTED)."""
        out = {}
        for i, g in enumerate(DISCONNECTED):
            s = (int(self.sum[i][1]) << 64) | int(self.sum[i][0])
            if s >> 127:
                s -= 1 << 128
            out[g] = (s, (int(self.sumsq[i][1]) << 64) | int(self.sumsq[i][0]))
        return out


class GsResultDisc(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double * 7), ("var", ctypes.c_double * 7),
                ("lb", ctypes.c_double * 7), ("ub", ctypes.c_double * 7),
                ("exact", ctypes.c_uint64 * 7), ("flags", ctypes.c_uint32 * 7)]

    def as_dict(self) -> dict:
        out = {}
        for i, g in enumerate(DISCONNECTED):
            f = int(self.flags[i])
            out[g] = {"X": self.x[i], "V": self.var[i], "lb": self.lb[i], "ub": self.ub[i],
                      "exact": int(self.exact[i]) if f & GS_F_EXACT and not f & GS_F_OVERFLOW
                      else None, "flags": f}
        return out


class GsResult(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double * 8), ("var", ctypes.c_double * 8),
                ("lb", ctypes.c_double * 8), ("ub", ctypes.c_double * 8),
                ("exact", ctypes.c_uint64 * 8), ("flags", ctypes.c_uint32 * 8)]

    def as_dict(self) -> dict:
        out = {}
        for i, g in enumerate(GRAPHLETS):
            f = int(self.flags[i])
            if not f & GS_F_COMPUTED:
                continue
            out[g] = {"X": self.x[i], "V": self.var[i], "lb": self.lb[i], "ub": self.ub[i],
                      "exact": int(self.exact[i]) if f & GS_F_EXACT and not f & GS_F_OVERFLOW
                      else None, "flags": f}
        return out


class GsStats(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("tri_tests", ctypes.c_int64),
                ("quad_tests", ctypes.c_int64), ("t_sum", ctypes.c_int64),
                ("tasks", ctypes.c_int64), ("model_bytes", ctypes.c_uint64),
                ("model_tri_bytes", ctypes.c_uint64), ("model_quad_bytes", ctypes.c_uint64),
                ("launches", ctypes.c_int64), ("launches_total", ctypes.c_int64),
                ("timed", ctypes.c_int32), ("ms_prep", ctypes.c_float), ("ms_tri", ctypes.c_float),
                ("ms_compact", ctypes.c_float), ("ms_cost", ctypes.c_float),
                ("ms_quad", ctypes.c_float), ("ms_fold", ctypes.c_float),
                ("dense_edges", ctypes.c_int64), ("dense_groups", ctypes.c_int64),
                ("micro_probes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class GsBatchStats(ctypes.Structure):
    _fields_ = [("num_graphs", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("tri_blocks_per_sm", ctypes.c_int32), ("quad_blocks_per_sm", ctypes.c_int32),
                ("task_probes", ctypes.c_int64), ("use_hubs", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_float),
                ("worst_ms", ctypes.c_float), ("graph_kernels", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


GS_BATCH_AUTOTUNE = 2


class GsRequest(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int32), ("mask", ctypes.c_uint32), ("fraction", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("z", ctypes.c_double)]


class GsRequestStats(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("batch_size", ctypes.c_int64), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("est_bytes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class GsServerStats(ctypes.Structure):
    _fields_ = [("graphs", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("peak_reserved_bytes", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_uint64), ("peak_in_flight", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib_handle = None


def lib() -> ctypes.CDLL:
    """The loaded libgraphlet.so; raises if it has not been built."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libgraphlet is not built ({_LIB_PATH} missing); run "
                           "paper_1701_01772_gb300.build() -- there is no CPU fallback")
    L = ctypes.CDLL(_LIB_PATH)
    P, I64, U64, U32, D = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                           ctypes.c_double)
    PP = ctypes.POINTER(ctypes.c_void_p)
    PI64 = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "gs_last_error": ([], ctypes.c_char_p),
        "gs_version": ([], ctypes.c_char_p),
        "gs_graph_create": ([P, P, I64, I64, U32, U64, P, PP], ctypes.c_int32),
        "gs_graph_destroy": ([P], ctypes.c_int32),
        "gs_graph_info": ([P, PI64, PI64, PI64, PI64, PI64], ctypes.c_int32),
        "gs_graph_index_info": ([P, PI64, PI64, PI64, PI64], ctypes.c_int32),
        "gs_count_adaptive": ([P, P, D, ctypes.c_int32, D, U64, U32, D, ctypes.POINTER(GsSums),
                               ctypes.POINTER(GsResult), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_double), P], ctypes.c_int32),
        "gs_per_edge_numerators": ([P, P, P, I64, P, P, P], ctypes.c_int32),
        "gs_sums_disc_merge": ([ctypes.POINTER(GsSumsDisc), ctypes.POINTER(GsSumsDisc)],
                               ctypes.c_int32),
        "gs_count_disconnected": ([P, P, P, I64, P, ctypes.POINTER(GsSumsDisc), P],
                                  ctypes.c_int32),
        "gs_estimate_disconnected": ([ctypes.POINTER(GsSumsDisc), D,
                                      ctypes.POINTER(GsResultDisc)], ctypes.c_int32),
        "gs_workspace_create": ([PP], ctypes.c_int32),
        "gs_workspace_destroy": ([P], ctypes.c_int32),
        "gs_workspace_bytes": ([P, ctypes.POINTER(U64)], ctypes.c_int32),
        "gs_sample": ([P, P, D, U64, P, I64, PI64, P], ctypes.c_int32),
        "gs_count": ([P, P, P, I64, U32, P, ctypes.POINTER(GsSums), P], ctypes.c_int32),
        "gs_estimate": ([ctypes.POINTER(GsSums), D, ctypes.POINTER(GsResult)], ctypes.c_int32),
        "gs_count_estimate": ([P, P, D, U64, U32, D, ctypes.POINTER(GsResult), PI64, P],
                              ctypes.c_int32),
        "gs_workspace_set_timing": ([P, ctypes.c_int], ctypes.c_int32),
        "gs_count3_static": ([P, P, I64, U32, ctypes.POINTER(GsSums), P], ctypes.c_int32),
        "gs_workspace_set_tuning": ([P, ctypes.c_int, ctypes.c_int, I64, ctypes.c_int],
                                    ctypes.c_int32),
        "gs_workspace_set_dense_slots": ([P, I64], ctypes.c_int32),
        "gs_sums_merge": ([ctypes.POINTER(GsSums), ctypes.POINTER(GsSums)], ctypes.c_int32),
        "gs_batch_create": ([P, P, P, I64, I64, I64, U32, U32, U64, P, PP], ctypes.c_int32),
        "gs_batch_count": ([P, ctypes.POINTER(GsSums), P], ctypes.c_int32),
        "gs_batch_info": ([P, ctypes.POINTER(GsBatchStats)], ctypes.c_int32),
        "gs_batch_destroy": ([P], ctypes.c_int32),
        "gs_server_create": ([U64, ctypes.c_int32, ctypes.c_int32, PP], ctypes.c_int32),
        "gs_server_add_graph": ([P, P, P, I64, I64, ctypes.POINTER(ctypes.c_int32)],
                                ctypes.c_int32),
        "gs_server_start": ([P, U32, U64, P], ctypes.c_int32),
        "gs_server_submit": ([P, ctypes.POINTER(GsRequest), ctypes.POINTER(U64)], ctypes.c_int32),
        "gs_server_wait": ([P, U64, D, ctypes.POINTER(GsResult), ctypes.POINTER(GsRequestStats)],
                           ctypes.c_int32),
        "gs_server_info": ([P, ctypes.POINTER(GsServerStats)], ctypes.c_int32),
        "gs_server_destroy": ([P], ctypes.c_int32),
        "gs_count_stats": ([P, ctypes.POINTER(GsStats)], ctypes.c_int32),
        "gs_sample_size": ([ctypes.POINTER(GsSums), D, D, PI64], ctypes.c_int32),
        "gs_core_numbers": ([P, P, P, ctypes.POINTER(ctypes.c_int32), P], ctypes.c_int32),
        "gs_sample_fixed": ([P, P, I64, U64, P, P], ctypes.c_int32),
        "gs_sample_ranks": ([P, P, I64, I64, U64, P, P], ctypes.c_int32),
        "gs_sample_weighted": ([P, P, P, D, U64, P, P, I64, PI64, ctypes.POINTER(ctypes.c_double),
                                P], ctypes.c_int32),
        "gs_count_weighted": ([P, P, P, I64, P, D, U32, D, ctypes.POINTER(GsResult), P],
                              ctypes.c_int32),
        "gs_micro": ([P, P, P, I64, D, U64, P, ctypes.POINTER(ctypes.c_double),
                      ctypes.POINTER(ctypes.c_int64), P], ctypes.c_int32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib_handle = L
    return L


def _check(status: int) -> None:
    if status != 0:
        msg = lib().gs_last_error()
        raise GraphletError(status, msg.decode() if msg else "")


def _stream_ptr(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _dev(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return t.data_ptr()


def _check_pairs(pairs, k: int) -> None:
    """A sampled-edge list is a [rows, 2] tensor holding at least k rows (the
    library reads exactly k pairs)."""
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must be a [k, 2] tensor")
    if not 0 <= k <= pairs.shape[0]:
        raise ValueError(f"k = {k} outside [0, {pairs.shape[0]}] (rows of pairs)")


# ------------------------------------------------------------------ C names

def gs_version() -> str:
    return lib().gs_version().decode()


def gs_graph_create(row_ptr, col, validate: bool = True, hub_budget_bytes: int = 0,
                    stream=None) -> int:
    import torch
    h = ctypes.c_void_p()
    n = row_ptr.numel() - 1
    _check(lib().gs_graph_create(_dev(row_ptr, torch.int64, "row_ptr"),
                                 _dev(col, torch.int32, "col") if col.numel() else None,
                                 n, col.numel(), GS_VALIDATE if validate else 0,
                                 hub_budget_bytes, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def gs_graph_destroy(handle: int) -> None:
    _check(lib().gs_graph_destroy(handle))


def gs_graph_info(handle: int) -> dict:
    vals = [ctypes.c_int64() for _ in range(5)]
    _check(lib().gs_graph_info(handle, *(ctypes.byref(v) for v in vals)))
    return dict(zip(("n", "m", "max_degree", "bitmap_hubs", "table_hubs"),
                    (v.value for v in vals)))


def gs_graph_index_info(handle: int) -> dict:
    vals = [ctypes.c_int64() for _ in range(4)]
    _check(lib().gs_graph_index_info(handle, *(ctypes.byref(v) for v in vals)))
    return dict(zip(("matrix_hubs", "mid_rows", "big_hubs", "dir_vertices"),
                    (v.value for v in vals)))


def gs_workspace_create() -> int:
    h = ctypes.c_void_p()
    _check(lib().gs_workspace_create(ctypes.byref(h)))
    return h.value


def gs_workspace_destroy(handle: int) -> None:
    _check(lib().gs_workspace_destroy(handle))


def gs_workspace_bytes(handle: int) -> int:
    v = ctypes.c_uint64()
    _check(lib().gs_workspace_bytes(handle, ctypes.byref(v)))
    return v.value


def gs_workspace_set_timing(handle: int, enable: bool) -> None:
    _check(lib().gs_workspace_set_timing(handle, int(enable)))


def gs_count_stats(handle: int) -> GsStats:
    out = GsStats()
    _check(lib().gs_count_stats(handle, ctypes.byref(out)))
    return out


def gs_sample(graph: int, ws: int, fraction: float, seed: int, out_pairs, stream=None) -> int:
    """Writes the sample into out_pairs (CUDA int32 [max_k, 2]); returns K."""
    import torch
    k = ctypes.c_int64()
    _check(lib().gs_sample(graph, ws, float(fraction), seed & (2**64 - 1),
                           _dev(out_pairs, torch.int32, "out_pairs"), out_pairs.shape[0],
                           ctypes.byref(k), _stream_ptr(stream)))
    return k.value


def gs_count(graph: int, ws: int, pairs, k: int, mask: int = GS_CONNECTED, per_edge=None,
             stream=None) -> GsSums:
    """pairs: CUDA int32 [k, 2] or None (all edges). per_edge: optional CUDA
    int64 [k, 3] receiving (t, k, q) per pair."""
    import torch
    if pairs is not None:
        _check_pairs(pairs, k)
    if per_edge is not None and (per_edge.dim() != 2 or per_edge.shape[1] != 3
                                 or per_edge.shape[0] < k):
        raise ValueError("per_edge must be a [>= k, 3] tensor")
    out = GsSums()
    _check(lib().gs_count(graph, ws, None if pairs is None else _dev(pairs, torch.int32, "pairs"),
                          k, mask,
                          None if per_edge is None else _dev(per_edge, torch.int64, "per_edge"),
                          ctypes.byref(out), _stream_ptr(stream)))
    return out


GS_STATIC_MAX_PAIRS = 1 << 20


def gs_count3_static(graph: int, pairs, k: int, mask: int = GS_THREE_NODE,
                     stream=None) -> GsSums:
    """Triangle / 2-star sums like gs_count, using only the library's fixed
    static scratch (no device allocation); k <= GS_STATIC_MAX_PAIRS. See
    include/graphlet.h for who needs it and its concurrency rules."""
    import torch
    if pairs is not None:
        _check_pairs(pairs, k)
    out = GsSums()
    _check(lib().gs_count3_static(graph, None if pairs is None else _dev(pairs, torch.int32, "pairs"),
                                  k, mask, ctypes.byref(out), _stream_ptr(stream)))
    return out


def gs_workspace_set_tuning(handle: int, tri_blocks_per_sm: int, quad_blocks_per_sm: int,
                            task_probes: int, use_hubs: bool) -> None:
    _check(lib().gs_workspace_set_tuning(handle, tri_blocks_per_sm, quad_blocks_per_sm,
                                         task_probes, int(use_hubs)))


def gs_workspace_set_dense_slots(handle: int, slots: int) -> None:
    _check(lib().gs_workspace_set_dense_slots(handle, slots))


def gs_batch_create(vtx_off, row_ptr, col, mask: int = GS_CONNECTED, flags: int = GS_VALIDATE,
                    hub_budget_bytes: int = 0, stream=None) -> int:
    """vtx_off: CUDA int64 [G+1]; row_ptr: CUDA int64 [N+1] (offsets into col);
    col: CUDA int32 [nnz] with graph-local ids."""
    import torch
    h = ctypes.c_void_p()
    _check(lib().gs_batch_create(_dev(vtx_off, torch.int64, "vtx_off"),
                                 _dev(row_ptr, torch.int64, "row_ptr"),
                                 _dev(col, torch.int32, "col") if col.numel() else None,
                                 vtx_off.numel() - 1, row_ptr.numel() - 1, col.numel(), mask, flags,
                                 hub_budget_bytes, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def gs_batch_count(handle: int, num_graphs: int, stream=None):
    out = (GsSums * num_graphs)()
    _check(lib().gs_batch_count(handle, out, _stream_ptr(stream)))
    return out


def gs_batch_info(handle: int) -> dict:
    out = GsBatchStats()
    _check(lib().gs_batch_info(handle, ctypes.byref(out)))
    return out.as_dict()


def gs_batch_destroy(handle: int) -> None:
    _check(lib().gs_batch_destroy(handle))


def gs_sums_merge(acc: GsSums, part: GsSums) -> GsSums:
    """acc += part (exact, host only), for shards of one sample."""
    _check(lib().gs_sums_merge(ctypes.byref(acc), ctypes.byref(part)))
    return acc


def sums_from_ints(k: int, m: int, mask: int, sums: dict, sq: dict) -> GsSums:
    """Packs exact Python-int sums {graphlet: value} into a GsSums."""
    out = GsSums()
    out.k, out.m, out.mask = k, m, mask
    for i, g in enumerate(GRAPHLETS):
        s = sums.get(g, 0) % (1 << 128)
        q = sq.get(g, 0)
        out.sum[i][0], out.sum[i][1] = s & (2**64 - 1), s >> 64
        out.sumsq[i][0], out.sumsq[i][1] = q & (2**64 - 1), q >> 64
    return out


def gs_estimate(sums: GsSums, z: float = 1.96) -> GsResult:
    out = GsResult()
    _check(lib().gs_estimate(ctypes.byref(sums), z, ctypes.byref(out)))
    return out


def gs_sample_size(sums: GsSums, rel_err: float, z: float = 1.96) -> dict:
    """Sample size per graphlet for a relative error of rel_err (host only)."""
    out = (ctypes.c_int64 * 8)()
    _check(lib().gs_sample_size(ctypes.byref(sums), float(z), float(rel_err), out))
    return {g: (None if out[i] < 0 else int(out[i])) for i, g in enumerate(GRAPHLETS)}


def gs_count_disconnected(graph: int, ws: int, pairs, k: int, per_edge, stream=None) -> GsSumsDisc:
    """pairs: CUDA int32 [k, 2], the list given to gs_count; per_edge: CUDA
    int64 [k, 3] that gs_count wrote for it with mask GS_CONNECTED."""
    import torch
    out = GsSumsDisc()
    _check(lib().gs_count_disconnected(graph, ws, _dev(pairs, torch.int32, "pairs"), k,
                                       _dev(per_edge, torch.int64, "per_edge"),
                                       ctypes.byref(out), _stream_ptr(stream)))
    return out


def gs_count_adaptive(graph: int, ws: int, beta: float, t_max: int = 20, phi: float = 0.0,
                      seed: int = 0, mask: int = GS_CONNECTED, z: float = 1.96, stream=None):
    """Algorithm 8: (sums, result, iterations, final fraction)."""
    sums, res = GsSums(), GsResult()
    iters, frac = ctypes.c_int32(), ctypes.c_double()
    _check(lib().gs_count_adaptive(graph, ws, float(beta), int(t_max), float(phi),
                                   seed & (2**64 - 1), mask, z, ctypes.byref(sums),
                                   ctypes.byref(res), ctypes.byref(iters), ctypes.byref(frac),
                                   _stream_ptr(stream)))
    return sums, res, iters.value, frac.value


def gs_per_edge_numerators(graph: int, ws: int, pairs, k: int, per_edge, out, stream=None) -> None:
    """out: CUDA int64 [k, 8] <- (N3, N4, N7, N8, N9, N10, N11, N12) per edge."""
    import torch
    _check(lib().gs_per_edge_numerators(graph, ws, _dev(pairs, torch.int32, "pairs"), k,
                                        _dev(per_edge, torch.int64, "per_edge"),
                                        _dev(out, torch.int64, "out"), _stream_ptr(stream)))


MICRO = tuple(range(3, 18))


def gs_sample_fixed(graph: int, ws: int, k: int, seed: int, out_pairs, stream=None):
    """Exactly k distinct uniform edges (smallest sampler keys) into
    out_pairs (CUDA int32 [>= k, 2]); returns out_pairs[:k]."""
    import torch
    if out_pairs.dim() != 2 or out_pairs.shape[1] != 2 or out_pairs.shape[0] < k:
        raise ValueError("out_pairs must be a [>= k, 2] tensor")
    _check(lib().gs_sample_fixed(graph, ws, int(k), seed & (2**64 - 1),
                                 _dev(out_pairs, torch.int32, "out_pairs"), _stream_ptr(stream)))
    return out_pairs[:k]


def gs_sample_ranks(graph: int, ws: int, k_lo: int, k_hi: int, seed: int, out_pairs,
                    stream=None):
    """Edges ranked [k_lo, k_hi) by sampler key into out_pairs (CUDA int32
    [>= k_hi - k_lo, 2]); returns out_pairs[:k_hi - k_lo]."""
    import torch
    k = k_hi - k_lo
    if out_pairs.dim() != 2 or out_pairs.shape[1] != 2 or out_pairs.shape[0] < k:
        raise ValueError("out_pairs must be a [>= k_hi - k_lo, 2] tensor")
    _check(lib().gs_sample_ranks(graph, ws, int(k_lo), int(k_hi), seed & (2**64 - 1),
                                 _dev(out_pairs, torch.int32, "out_pairs"), _stream_ptr(stream)))
    return out_pairs[:k]


def gs_core_numbers(graph: int, ws: int, out, stream=None) -> int:
    """out (CUDA int32 [n]) <- k-core number per vertex; returns the largest."""
    import torch
    mx = ctypes.c_int32()
    _check(lib().gs_core_numbers(graph, ws, _dev(out, torch.int32, "out"), ctypes.byref(mx),
                                 _stream_ptr(stream)))
    return mx.value


def gs_sample_weighted(graph: int, ws: int, vertex_w, fraction: float, seed: int, out_pairs,
                       out_w=None, stream=None):
    """Weighted edge sample into out_pairs (CUDA int32 [max_k, 2]) and out_w
    (CUDA int32 [max_k] or None); returns (K, scale s)."""
    import torch
    k = ctypes.c_int64()
    sc = ctypes.c_double()
    _check(lib().gs_sample_weighted(graph, ws, _dev(vertex_w, torch.int32, "vertex_w"),
                                    float(fraction), seed & (2**64 - 1),
                                    _dev(out_pairs, torch.int32, "out_pairs"),
                                    None if out_w is None else _dev(out_w, torch.int32, "out_w"),
                                    out_pairs.shape[0], ctypes.byref(k), ctypes.byref(sc),
                                    _stream_ptr(stream)))
    return k.value, sc.value


def gs_count_weighted(graph: int, ws: int, pairs, k: int, vertex_w, scale: float,
                      mask: int = GS_CONNECTED, z: float = 1.96, stream=None) -> GsResult:
    """Horvitz-Thompson estimates of a weighted sample (sigma_e = 1 / pi_e)."""
    import torch
    _check_pairs(pairs, k)
    out = GsResult()
    _check(lib().gs_count_weighted(graph, ws, _dev(pairs, torch.int32, "pairs"), k,
                                   _dev(vertex_w, torch.int32, "vertex_w"), float(scale), mask,
                                   z, ctypes.byref(out), _stream_ptr(stream)))
    return out


def gs_micro(graph: int, ws: int, pairs, k: int, p_e: float, seed: int, out, stream=None):
    """Algorithm 7: out (CUDA float64 [k, 15]) <- x3..x17 per sampled edge.
    Returns (max per statistic, first edge index holding it) over the
    sample (Sec. 7's extremal statistic)."""
    import torch
    _check_pairs(pairs, k)
    if out.dim() != 2 or out.shape[1] != 15 or out.shape[0] < k:
        raise ValueError("out must be a [>= k, 15] float64 tensor")
    mx = (ctypes.c_double * 15)()
    arg = (ctypes.c_int64 * 15)()
    _check(lib().gs_micro(graph, ws, _dev(pairs, torch.int32, "pairs"), k, float(p_e),
                          seed & (2**64 - 1), _dev(out, torch.float64, "out"), mx, arg,
                          _stream_ptr(stream)))
    return list(mx), list(arg)


def disc_sums_from_ints(k: int, m: int, n: int, sums: dict, sq: dict) -> GsSumsDisc:
    """Packs exact Python-int sums {graphlet: value} (graphlets of DISCONNECTED)
    into a GsSumsDisc."""
    out = GsSumsDisc()
    out.k, out.m, out.n = k, m, n
    for i, g in enumerate(DISCONNECTED):
        s = sums.get(g, 0) % (1 << 128)
        q = sq.get(g, 0)
        out.sum[i][0], out.sum[i][1] = s & (2**64 - 1), s >> 64
        out.sumsq[i][0], out.sumsq[i][1] = q & (2**64 - 1), q >> 64
    return out


def gs_sums_disc_merge(acc: GsSumsDisc, part: GsSumsDisc) -> GsSumsDisc:
    out = GsSumsDisc.from_buffer_copy(acc)
    _check(lib().gs_sums_disc_merge(ctypes.byref(out), ctypes.byref(part)))
    return out


def gs_estimate_disconnected(sums: GsSumsDisc, z: float = 1.96) -> GsResultDisc:
    out = GsResultDisc()
    _check(lib().gs_estimate_disconnected(ctypes.byref(sums), z, ctypes.byref(out)))
    return out


def gs_count_estimate(graph: int, ws: int, fraction: float, seed: int,
                      mask: int = GS_CONNECTED, z: float = 1.96, stream=None):
    out = GsResult()
    k = ctypes.c_int64()
    _check(lib().gs_count_estimate(graph, ws, float(fraction), seed & (2**64 - 1), mask, z,
                                   ctypes.byref(out), ctypes.byref(k), _stream_ptr(stream)))
    return out, k.value


# ------------------------------------------------------------------ owners

class Workspace:
    def __init__(self):
        self.handle = gs_workspace_create()

    def nbytes(self) -> int:
        return gs_workspace_bytes(self.handle)

    def set_timing(self, enable: bool = True) -> None:
        gs_workspace_set_timing(self.handle, enable)

    def set_tuning(self, tri_blocks_per_sm: int = 8, quad_blocks_per_sm: int = 8,
                   task_probes: int = 512, use_hubs: bool = True) -> None:
        gs_workspace_set_tuning(self.handle, tri_blocks_per_sm, quad_blocks_per_sm, task_probes,
                                use_hubs)

    def set_dense_slots(self, slots: int) -> None:
        gs_workspace_set_dense_slots(self.handle, slots)

    def stats(self) -> dict:
        return gs_count_stats(self.handle).as_dict()

    def close(self):
        if self.handle:
            gs_workspace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A registered CSR graph (keeps the device tensors alive)."""

    def __init__(self, row_ptr, col, validate: bool = True, hub_budget_bytes: int = 0,
                 stream=None):
        self.row_ptr, self.col = row_ptr, col
        self.handle = gs_graph_create(row_ptr, col, validate, hub_budget_bytes, stream)
        self.info = gs_graph_info(self.handle)
        self.info.update(gs_graph_index_info(self.handle))
        self.ws = Workspace()

    @classmethod
    def from_numpy(cls, row_ptr, col, device="cuda", **kw):
        import torch
        return cls(torch.as_tensor(row_ptr, dtype=torch.int64).to(device),
                   torch.as_tensor(col, dtype=torch.int32).to(device), **kw)

    @property
    def m(self) -> int:
        return self.info["m"]

    def sample(self, fraction: float, seed: int, stream=None):
        import torch
        cap = max(1, int(self.m * fraction * 1.2 + 10 * math.sqrt(self.m * fraction + 1) + 64))
        cap = min(cap, max(self.m, 1))
        while True:
            out = torch.empty((cap, 2), dtype=torch.int32, device=self.row_ptr.device)
            try:
                k = gs_sample(self.handle, self.ws.handle, fraction, seed, out, stream)
                return out[:k]
            except GraphletError as e:
                if e.status != 13 or cap >= self.m:
                    raise
                cap = self.m

    def count(self, pairs=None, mask: int = GS_CONNECTED, per_edge=None, stream=None) -> GsSums:
        k = self.m if pairs is None else pairs.shape[0]
        return gs_count(self.handle, self.ws.handle, pairs, k, mask, per_edge, stream)

    def count_all(self, pairs=None, stream=None):
        """Connected and disconnected sums of one sampled-edge list (None: every
        edge, listed by the sampler at fraction 1): (GsSums, GsSumsDisc)."""
        import torch
        if pairs is None:
            pairs = self.sample(1.0, 0)
        k = pairs.shape[0]
        per = torch.empty((k, 3), dtype=torch.int64, device=pairs.device)
        conn = gs_count(self.handle, self.ws.handle, pairs, k, GS_CONNECTED, per, stream)
        disc = gs_count_disconnected(self.handle, self.ws.handle, pairs, k, per, stream)
        return conn, disc

    def count_estimate(self, fraction: float, seed: int = 0, mask: int = GS_CONNECTED,
                       z: float = 1.96, stream=None):
        return gs_count_estimate(self.handle, self.ws.handle, fraction, seed, mask, z, stream)

    def close(self):
        if getattr(self, "ws", None) is not None:
            self.ws.close()
        if getattr(self, "handle", None):
            gs_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many small graphs counted exactly in one CUDA-graph launch."""

    def __init__(self, vtx_off, row_ptr, col, mask: int = GS_CONNECTED, autotune: bool = True,
                 validate: bool = True, hub_budget_bytes: int = 0, stream=None):
        self.vtx_off, self.row_ptr, self.col = vtx_off, row_ptr, col
        self.num_graphs = vtx_off.numel() - 1
        flags = (GS_VALIDATE if validate else 0) | (GS_BATCH_AUTOTUNE if autotune else 0)
        self.handle = gs_batch_create(vtx_off, row_ptr, col, mask, flags, hub_budget_bytes, stream)

    @classmethod
    def from_graphs(cls, graphs, device="cuda", **kw):
        """graphs: list of (row_ptr, col) numpy arrays (local ids)."""
        import numpy as np
        import torch
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
        t = lambda a, dt: torch.as_tensor(a, dtype=dt).to(device)  # noqa: E731
        return cls(t(vtx_off, torch.int64), t(row_ptr, torch.int64), t(col, torch.int32), **kw)

    def count(self, stream=None):
        return gs_batch_count(self.handle, self.num_graphs, stream)

    def exact(self, stream=None) -> list:
        """Exact counts {graphlet: count} per graph."""
        out = []
        for s in self.count(stream):
            r = gs_estimate(s).as_dict()
            out.append({g: r[g]["exact"] if s.k > 0 else 0 for g in r})
        return out

    def info(self) -> dict:
        return gs_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            gs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

def gs_server_create(hbm_budget_bytes: int, max_batch: int = 64, lanes: int = 2) -> int:
    h = ctypes.c_void_p()
    _check(lib().gs_server_create(hbm_budget_bytes, max_batch, lanes, ctypes.byref(h)))
    return h.value


def gs_server_add_graph(server: int, row_ptr, col) -> int:
    import torch
    gid = ctypes.c_int32()
    _check(lib().gs_server_add_graph(server, _dev(row_ptr, torch.int64, "row_ptr"),
                                     _dev(col, torch.int32, "col") if col.numel() else None,
                                     row_ptr.numel() - 1, col.numel(), ctypes.byref(gid)))
    return gid.value


def gs_server_start(server: int, validate: bool = True, hub_budget_bytes: int = 0,
                    stream=None) -> None:
    _check(lib().gs_server_start(server, GS_VALIDATE if validate else 0, hub_budget_bytes,
                                 _stream_ptr(stream)))


def gs_server_submit(server: int, graph: int, fraction: float, seed: int,
                     mask: int = GS_CONNECTED, z: float = 1.96) -> int:
    req = GsRequest(graph, mask, float(fraction), seed & (2**64 - 1), z)
    t = ctypes.c_uint64()
    _check(lib().gs_server_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def gs_server_wait(server: int, ticket: int, timeout_s: float = 600.0):
    res = GsResult()
    st = GsRequestStats()
    _check(lib().gs_server_wait(server, ticket, timeout_s, ctypes.byref(res), ctypes.byref(st)))
    return res, st.as_dict()


def gs_server_info(server: int) -> dict:
    out = GsServerStats()
    _check(lib().gs_server_info(server, ctypes.byref(out)))
    return out.as_dict()


def gs_server_destroy(server: int) -> None:
    _check(lib().gs_server_destroy(server))


class Server:
    """Continuous-batching estimation server over resident graphs."""

    def __init__(self, hbm_budget_bytes: int = 40 << 30, max_batch: int = 64, lanes: int = 2):
        self.handle = gs_server_create(hbm_budget_bytes, max_batch, lanes)
        self._keep = []

    def add_graph(self, row_ptr, col) -> int:
        self._keep.append((row_ptr, col))
        return gs_server_add_graph(self.handle, row_ptr, col)

    def add_numpy(self, row_ptr, col, device="cuda") -> int:
        import torch
        return self.add_graph(torch.as_tensor(row_ptr, dtype=torch.int64).to(device),
                              torch.as_tensor(col, dtype=torch.int32).to(device))

    def start(self, validate: bool = True, hub_budget_bytes: int = 0):
        gs_server_start(self.handle, validate, hub_budget_bytes)

    def submit(self, graph: int, fraction: float, seed: int, mask: int = GS_CONNECTED,
               z: float = 1.96) -> int:
        return gs_server_submit(self.handle, graph, fraction, seed, mask, z)

    def wait(self, ticket: int, timeout_s: float = 600.0):
        return gs_server_wait(self.handle, ticket, timeout_s)

    def info(self) -> dict:
        return gs_server_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            gs_server_destroy(self.handle)
            self.handle = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
