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

STATUS = {0: "GS_OK", 1: "GS_EINVAL", 2: "GS_ENOTSORTED", 3: "GS_ESELFLOOP", 4: "GS_EDUP",
          5: "GS_EASYM", 6: "GS_EEDGE", 7: "GS_EDUPSAMPLE", 8: "GS_EOVERFLOW", 9: "GS_ENOMEM",
          10: "GS_EBUDGET", 11: "GS_ETIMEOUT", 12: "GS_ECUDA", 13: "GS_ECAPACITY"}


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
                ("ms_quad", ctypes.c_float), ("ms_fold", ctypes.c_float)]

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
        "gs_count_stats": ([P, ctypes.POINTER(GsStats)], ctypes.c_int32),
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
    out = GsSums()
    _check(lib().gs_count3_static(graph, None if pairs is None else _dev(pairs, torch.int32, "pairs"),
                                  k, mask, ctypes.byref(out), _stream_ptr(stream)))
    return out


def gs_estimate(sums: GsSums, z: float = 1.96) -> GsResult:
    out = GsResult()
    _check(lib().gs_estimate(ctypes.byref(sums), z, ctypes.byref(out)))
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
