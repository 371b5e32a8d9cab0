#!/usr/bin/env python
"""Benchmark: sampled edges/s for connected 3- and 4-node graphlet estimation.

Headline workload (the largest configuration that fits one GPU): R-MAT scale
24, edge factor 16, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), symmetrised,
deduplicated, self-loops removed (16,777,216 vertices, 260,388,226 edges).
One step = exact 3-node counts over every edge, then 4-node estimates (all
connected graphlets, with variances and 95% bounds) on seeded edge samples of
0.1% and 1% drawn by the library's sampler on the device.
value = edges processed / device time. The 1M-vertex Chung-Lu configuration
(fractions 1%, 5%, 10% and exact) is measured after it and reported under
"extra".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--workload rmat_24|chung_lu_1m|batch|serve]

Under torchrun (N > 1) every rank runs the same step with its own seeds on its
own GPU (weak scaling, no data-path collective); the time is the max over
ranks. --impl reference times the CPU oracle on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sampled edges/s for 4-node graphlet counts; p50/p99 estimate latency"
UNIT = "edges/s"
THREE, CONN = (1 << 3) | (1 << 4), sum(1 << b for b in (3, 4, 7, 8, 9, 10, 11, 12))

# workload name -> (description, [(label, fraction, mask)])
WORKLOADS = {
    "rmat_24": (
        "rmat_24: R-MAT scale 24, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
        "symmetrised, deduplicated, self-loops removed (16,777,216 vertices, 260,388,226 "
        "edges), int32 CSR; exact 3-node counts (G3, G4) over all edges plus 4-node "
        "estimates (G3, G4, G7-G12) at 0.1% and 1% edge samples (seeded, library sampler)",
        [("exact_3node", 1.0, THREE), ("0.001", 0.001, CONN), ("0.01", 0.01, CONN)]),
    "rmat_22": (
        "rmat_22: R-MAT scale 22, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
        "symmetrised, deduplicated, self-loops removed (4,194,304 vertices), int32 CSR; the "
        "headline's parts on a graph small enough for full ncu counter captures",
        [("exact_3node", 1.0, THREE), ("0.001", 0.001, CONN), ("0.01", 0.01, CONN)]),
    "chung_lu_1m": (
        "chung_lu_1m: Chung-Lu n=1,000,000, m~20M, degree exponent 2.1, expected degree "
        "cap 50,000, int32 CSR; edge-sample fractions 1%, 5%, 10% (seeded, library sampler) "
        "plus exact counts at fraction 1; graphlets G3,G4,G7-G12",
        [("0.01", 0.01, CONN), ("0.05", 0.05, CONN), ("0.1", 0.10, CONN), ("exact", 1.0, CONN)]),
}
# algorithmic bytes of the 4-node phase: a membership test reads one 4-byte
# element of the iterated list and one 4-byte word (bitmap or matrix word,
# directory entry, list entry) that answers it; a dense-edge matrix group
# reads one 16-byte group of a hub-matrix row (the edge's T-mask group it is
# ANDed with sits in shared memory)
BYTES_PER_TEST = 8
BYTES_PER_DENSE_GROUP = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--hub-budget", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the Chung-Lu 1M measurement after the headline")
    ap.add_argument("--extra-steps", type=int, default=5)
    ap.add_argument("--workload", choices=("rmat_24", "rmat_22", "chung_lu_1m", "batch", "serve"),
                    default="rmat_24",
                    help="rmat_24 = the headline line; chung_lu_1m alone; rmat_22 = the small "
                         "case for counter captures; batch / serve = the batched and served "
                         "paths against one plain launch per graph / request")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-loads", type=str, default="0.3,0.6,0.9",
                    help="offered loads as fractions of the measured capacity")
    return ap.parse_args()


def generate(name):
    import synth
    if name == "rmat_24":
        return synth.rmat_24()
    if name == "rmat_22":
        return synth.rmat(22, 16, synth.BASE_SEED + 2)
    return synth.chung_lu_1m()


# ------------------------------------------------------------------ helpers

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the 4-node kernels' source and of the index they read (its
    build in graph.cu), with comments and blank space removed, so that a
    comment edit does not invalidate recorded counters."""
    import re
    h = hashlib.sha256()
    for name in ("count.cu", "common.cuh", "graph.cu"):
        with open(os.path.join(ROOT, "paper_1701_01772_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def load_traffic(key: str):
    """DRAM bytes per test from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        rec = t.get(key)
        if rec and rec.get("source_hash") == kernel_source_hash():
            return rec
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for name, val in zip(names, p[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * p / 100.0
    lo, hi = int(k), min(int(k) + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


# ------------------------------------------------------------------ GPU arm

def incidences_from_numerators(n: dict) -> int:
    """Connected 3- and 4-node graphlet incidences of the counted edges,
    sum over e of t + a + b + k + C(t,2) + t(a+b) + q + C(a,2) + C(b,2) + ab,
    from the exact numerator sums {i: sum N_i}: N3 + N4 + 2 N7 + 5 N8
    + (3 N9 + N11) / 2 + 2 N10 + N12, where per edge
    (3 N9 + N11) / 2 = t(a+b) - 4 N8 + C(a,2) + C(b,2) is an integer.
    Graphlets outside the mask count 0."""
    g = lambda i: n.get(i, 0)  # noqa: E731
    return (g(3) + g(4) + 2 * g(7) + 5 * g(8) + (3 * g(9) + g(11)) // 2 + 2 * g(10) + g(12))


def run_gpu(args, rank, world, device, name, rp, col, steps, warmup):
    import torch

    import paper_1701_01772_gb300 as gs

    torch.cuda.set_device(device)
    gs.build()
    desc, parts = WORKLOADS[name]
    dev = f"cuda:{device}"
    row_ptr = torch.as_tensor(rp, device=dev)
    colt = torch.as_tensor(col, device=dev)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    t0 = time.perf_counter()
    g = gs.Graph(row_ptr, colt, hub_budget_bytes=args.hub_budget)
    torch.cuda.synchronize()
    registration_s = time.perf_counter() - t0
    free1, _ = torch.cuda.mem_get_info()
    index_bytes = free0 - free1
    ws = g.ws
    ws.set_timing(True)
    stream = torch.cuda.current_stream()
    m = g.m
    sampled = [f for _, f, _ in parts if f < 1.0]
    cap = int(max(sampled) * m * 1.05) + 1024 if sampled else 1
    pair_buf = torch.empty((min(cap, m), 2), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def seed_of(step, fi):
        return (rank * 1_000_003 + step * 101 + fi * 7 + 1) & (2**63 - 1)

    part_stats = {}

    def one_step(step):
        """Every part of the workload: sample (fraction < 1) + count +
        estimate. Returns (edges, [(label, ms)], [(stats)], incidences)."""
        edges, lat, quad, inc = 0, [], [], 0
        for fi, (label, f, mask) in enumerate(parts):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            if f >= 1.0:
                sums = gs.gs_count(g.handle, ws.handle, None, m, mask)
                k = m
            else:
                k = gs.gs_sample(g.handle, ws.handle, f, seed_of(step, fi), pair_buf)
                sums = gs.gs_count(g.handle, ws.handle, pair_buf[:k], k, mask)
            gs.gs_estimate(sums)
            ev1.record(stream)
            st = gs.gs_count_stats(ws.handle)
            torch.cuda.synchronize()
            lat.append((label, ev0.elapsed_time(ev1)))
            quad.append((st.ms_quad, st.quad_tests - st.dense_groups, st.dense_groups,
                         st.model_quad_bytes))
            part_stats[label] = {"K": k, "tri_tests": st.tri_tests, "ms_tri": round(st.ms_tri, 3),
                                 "quad_tests": st.quad_tests - st.dense_groups,
                                 "dense_groups": st.dense_groups, "ms_quad": round(st.ms_quad, 3),
                                 "ms_cost": round(st.ms_cost, 3)}
            edges += k
            inc += incidences_from_numerators({gid: v[0] for gid, v in sums.sums().items()})
        return edges, lat, quad, inc

    for w in range(warmup):
        flush.fill_(w & 0xFF)
        one_step(10_000 + w)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_edges, total_ms, total_inc = 0, 0.0, 0
    lat_by = {label: [] for label, _, _ in parts}
    quad_ms, tests, groups, model_bytes, quad_launches = 0.0, 0, 0, 0, 0
    units_by = {}  # 4-node units (tests + dense groups) per part label
    launches0 = gs.gs_count_stats(ws.handle).launches_total
    with ClockSampler(device) as clocks:
        for step in range(steps):
            flush.fill_((step + 1) & 0xFF)  # L2 flush, outside the timed events
            torch.cuda.synchronize()
            e, lat, quad, inc = one_step(step)
            total_edges += e
            total_inc += inc
            total_ms += sum(ms for _, ms in lat)
            for label, ms in lat:
                lat_by[label].append(ms)
            for (label, _), (qms, qt, qg, qb) in zip(lat, quad):
                if qms > 0:
                    quad_ms += qms
                    tests += qt
                    groups += qg
                    model_bytes += qb
                    quad_launches += 1
                    units_by[label] = units_by.get(label, 0) + qt + qg
    torch.cuda.synchronize()
    launches = gs.gs_count_stats(ws.handle).launches_total - launches0
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e = torch.tensor([total_edges, total_inc], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(e, op=torch.distributed.ReduceOp.SUM)
        total_ms_max, edges_all, inc_all = float(t.item()), int(e[0].item()), float(e[1].item())
    else:
        total_ms_max, edges_all, inc_all = total_ms, total_edges, float(total_inc)

    # ---- end to end through the C ABI with host buffers: each sampled
    # part's explicit edge list is copied from pinned host memory, counted
    # and estimated; the sums come back to the host. The exact pass names
    # the resident graph's own edges (no input copy).
    host_lists = []
    for fi, (label, f, mask) in enumerate(parts):
        if f >= 1.0:
            host_lists.append((None, mask))
        else:
            k = gs.gs_sample(g.handle, ws.handle, f, seed_of(5000, fi), pair_buf)
            host_lists.append((pair_buf[:k].cpu().pin_memory(), mask))
    dev_buf = torch.empty_like(pair_buf)
    e2e_edges, e2e_ms, h2d, d2h = 0, 0.0, 0, 0
    e2e_steps = max(1, min(steps, 5))  # the same step, repeated at most 5 times
    for step in range(e2e_steps):
        flush.fill_((step + 7) & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for hl, mask in host_lists:
            if hl is None:
                sums = gs.gs_count(g.handle, ws.handle, None, m, mask)
                e2e_edges += m
            else:
                k = hl.shape[0]
                dev_buf[:k].copy_(hl, non_blocking=True)
                sums = gs.gs_count(g.handle, ws.handle, dev_buf[:k], k, mask)
                e2e_edges += k
                h2d += hl.numel() * 4
            gs.gs_estimate(sums)
            d2h += 280  # gs_sums returned to the host
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e = {"value": e2e_edges / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps,
           "steps": e2e_steps}

    peak, peak_kind = load_peaks()
    alg_bytes = BYTES_PER_TEST * tests + BYTES_PER_DENSE_GROUP * groups
    secs = quad_ms / 1e3
    achieved = alg_bytes / secs / 1e9 if secs > 0 else 0.0
    traffic = load_traffic(f"quad_phase_{name}")
    traffic_bytes = None
    if traffic:
        # DRAM bytes per unit measured per sample fraction on the small case
        # (a larger sample reuses more of L2), applied to each part's units
        bpu = traffic["dram_bytes_per_unit"]
        traffic_bytes = sum(units * bpu.get(label, bpu["default"])
                            for label, units in units_by.items()) / max(quad_launches, 1)
    avg_s = secs / max(quad_launches, 1)
    roofline = {
        "kernel": "4-node phase: k_quad (membership tests) + k_dense_pairs (dense-edge "
                  "member pairs), all 4-node launches of the timed steps",
        "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
        "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
        "bytes_model": f"{BYTES_PER_TEST} B per membership test + {BYTES_PER_DENSE_GROUP} B per "
                       "128-bit dense group",
        "traffic": round(traffic_bytes) if traffic_bytes else None,
        "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of k_quad + "
                           "k_dense_pairs per unit on a small case at the same sample "
                           "fractions, x each part's units")
        if traffic else None,
        "dram_frac": round(traffic_bytes / avg_s / 1e9 / peak, 4) if traffic_bytes else None,
        "avg_launch_ms": round(quad_ms / max(quad_launches, 1), 3),
        "tests_per_launch": round(tests / max(quad_launches, 1)),
        "dense_groups_per_launch": round(groups / max(quad_launches, 1)),
        "tests_per_s": round((tests + groups) / secs, 1) if secs > 0 else None,
        "model_bytes_avoided_per_launch": model_bytes // max(quad_launches, 1),
    }
    out = {
        "desc": desc, "edges_all": edges_all, "ms_total": total_ms_max, "inc_all": inc_all,
        "lat": {label: {"p50_ms": round(percentile(v, 50), 3),
                        "p99_ms": round(percentile(v, 99), 3)} for label, v in lat_by.items()},
        "e2e": e2e, "roofline": roofline, "launches": launches, "clocks": clocks.summary(),
        "graph": g.info, "parts": [label for label, _, _ in parts],
        "registration_s": round(registration_s, 3), "index_bytes": int(index_bytes),
        "workspace_bytes": int(ws.nbytes()), "part_stats": part_stats,
    }
    g.close()
    del pair_buf, flush, dev_buf, row_ptr, colt
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ oracle arm

def _oracle_worker_init(rp_path, col_path):
    global _ORACLE_CSR
    import numpy as np
    sys.path.insert(0, ROOT)
    _ORACLE_CSR = (np.load(rp_path, mmap_mode="r"), np.load(col_path, mmap_mode="r"))


_ORACLE_CSR = None


def _oracle_worker_chunk(job):
    """Per-edge local counts of one chunk of sampled edges by the oracle;
    returns the chunk's exact numerator sums."""
    import numpy as np
    import oracle
    chunk, four = job
    rp, col = _ORACLE_CSR
    lc = oracle.local_counts(np.asarray(rp), np.asarray(col), chunk, four=four)
    return oracle.numerators(lc)


class OraclePool:
    """One spawned process per host core, each holding the CSR through
    memory-mapped .npy files (written once)."""

    def __init__(self, rp, col, workers=None):
        import multiprocessing as mp
        import tempfile

        import numpy as np
        self.workers = workers or os.cpu_count() or 1
        self.tmp = tempfile.mkdtemp(prefix="gs_oracle_")
        self.paths = (os.path.join(self.tmp, "rp.npy"), os.path.join(self.tmp, "col.npy"))
        np.save(self.paths[0], rp)
        np.save(self.paths[1], col)
        self.pool = mp.get_context("spawn").Pool(self.workers, _oracle_worker_init, self.paths)

    def close(self):
        self.pool.close()
        self.pool.join()
        for f in self.paths:
            os.remove(f)
        os.rmdir(self.tmp)


def oracle_part_rates(rp, col, parts, seconds: float, seed: int = 1, workers: int | None = None,
                      pool: OraclePool | None = None):
    """The CPU oracle, unchanged, run by one spawned process per host core
    over disjoint chunks of each part's edges (the first edges of a seeded
    sample at that part's fraction; all edges in canonical order for the
    exact part): each part gets `seconds` / len(parts) of wall time, sized
    by a single-core calibration pass. Returns ({label: (edges, wall s)},
    cores)."""
    import oracle
    import synth
    own = pool is None
    if own:
        pool = OraclePool(rp, col, workers)
    budget = seconds / max(len(parts), 1)
    rates = {}
    try:
        for label, f, mask in parts:
            four = bool(mask & ~THREE)
            if f >= 1.0:
                pairs = synth.upper_pairs(rp, col)[: max(1, 400_000 * pool.workers)]
            else:
                pairs = oracle.sample(rp, col, f, seed)
            # single-core calibration
            n, used, done = 16, 0.0, 0
            while done < len(pairs) and used < max(0.3, budget / 8):
                t0 = time.process_time()
                oracle.numerators(oracle.local_counts(rp, col, pairs[done:done + n], four=four))
                used += time.process_time() - t0
                done += n
                n = min(2 * n, 65536)
            per_core = max(16, int(done / max(used, 1e-6) * budget))
            total = min(len(pairs), per_core * pool.workers)
            step = max(1, total // (4 * pool.workers))
            jobs = [(pairs[i:i + step], four) for i in range(0, total, step)]
            pool.pool.map(_oracle_worker_chunk, [(pairs[:pool.workers], four)], chunksize=1)
            t0 = time.perf_counter()
            pool.pool.map(_oracle_worker_chunk, jobs, chunksize=1)
            rates[label] = (total, time.perf_counter() - t0)
    finally:
        if own:
            pool.close()
    return rates, pool.workers


def oracle_step_rate(rp, col, parts, seconds, seed=1, pool=None):
    """Edges/s of the oracle on one whole step of the workload: each part's
    measured per-edge rate applied to that part's full edge count."""
    m = len(col) // 2
    rates, cores = oracle_part_rates(rp, col, parts, seconds, seed, pool=pool)
    step_edges = sum(m if f >= 1.0 else f * m for _, f, _ in parts)
    step_secs = sum((m if f >= 1.0 else f * m) * rates[label][1] / max(rates[label][0], 1)
                    for label, f, _ in parts)
    sample = "; ".join(f"{label}: {rates[label][0]} edges in {rates[label][1]:.1f} s"
                       for label, _, _ in parts)
    return step_edges / step_secs, cores, sample, sum(r[1] for r in rates.values())


def run_reference(args, rank, world):
    if rank != 0:
        return None
    name = "chung_lu_1m" if args.workload == "chung_lu_1m" else "rmat_24"
    desc, parts = WORKLOADS[name]
    rp, col = generate(name)
    budget = max(6.0, min(45.0, 150.0 / max(args.steps + args.warmup, 1)))
    values, walls, cores, sample = [], 0.0, 1, ""
    pool = OraclePool(rp, col)
    try:
        for step in range(args.warmup + args.steps):
            v, cores, sample, wall = oracle_step_rate(rp, col, parts, budget, seed=1 + step,
                                                      pool=pool)
            if step >= args.warmup:
                values.append(v)
                walls += wall
    finally:
        pool.close()
    value = statistics.median(values)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": walls * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": desc,
                   "sample": "bounded: per step, the first edges of each part (seeded sample "
                             "or canonical edge order), per-edge rates scaled to the full step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"last step: {sample}; one spawned process per core"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------------ batched

def run_batch_bench(args):
    """4096 small graphs (n ~ U{50..5000}, mean degree ~ U[4,40], ER /
    Chung-Lu 2.3 / 2-D RGG): exact connected counts for every graph in one
    CUDA-graph launch, against one gs_count per graph (each graph registered
    beforehand, counting only in the timed region)."""
    import numpy as np
    import torch

    import paper_1701_01772_gb300 as gs
    import synth

    gs.build()
    t0 = time.time()
    graphs = synth.batch_4096(args.batch_graphs)
    gen_s = time.time() - t0
    edges = sum(len(c) // 2 for _, c in graphs)
    t0 = time.time()
    b = gs.Batch.from_graphs(graphs, autotune=True)
    create_s = time.time() - t0
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.count()
    ms = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sums = b.count()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    batched_ms = statistics.median(ms)
    # baseline: one plain gs_count launch sequence per graph
    # (small per-graph hub index: 4096 full-size co-degree tables would not fit)
    singles = [gs.Graph.from_numpy(rp, col, hub_budget_bytes=1 << 20) for rp, col in graphs]
    for g in singles[:8]:
        g.count(None, gs.GS_CONNECTED)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    per_graph = [g.count(None, gs.GS_CONNECTED) for g in singles]
    e1.record(stream)
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1)
    same = all(a.sums() == c.sums() for a, c in zip(sums, per_graph))
    info = b.info()
    for g in singles:
        g.close()
    b.close()
    return {
        "metric": "graphs/s for exact connected 3- and 4-node counts (batched)",
        "value": round(len(graphs) / (batched_ms / 1e3), 1), "unit": "graphs/s",
        "edges_per_s": round(edges / (batched_ms / 1e3), 1),
        "ms_per_step": round(batched_ms, 3), "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"batch: {len(graphs)} graphs, {edges} edges, n ~ U{{50..5000}}, "
                               "mean degree ~ U[4,40], ER / Chung-Lu 2.3 / RGG",
                   "generation_s": round(gen_s, 1), "create_and_autotune_s": round(create_s, 2)},
        "autotune": info,
        "baseline_one_launch_per_graph_ms": round(single_ms, 3),
        "speedup_vs_per_graph": round(single_ms / batched_ms, 2),
        "identical_results": same,
    }


# ------------------------------------------------------------------ serving

def run_serve_bench(args):
    """Serving: 8 resident graphs (ER 2000 x2, Chung-Lu 100k x2, Chung-Lu 1M
    x2, R-MAT 24 x2); each request names a graph, a fraction log-uniform in
    [0.1%, 10%], a seed and a random non-empty graphlet mask (3-node masks
    only on the R-MAT graphs: a 4-node R-MAT request takes about 0.7 s per
    0.1% of its edges, up to 70 s at 10%, four orders of magnitude beyond
    the offered rate). The capacity of one launch per request (requests run
    one by one with gs_count_estimate) is measured first; then open-loop
    Poisson streams at 30%, 60% and 90% of it, and at the offered 2000
    req/s, run through the server (40 GB budget, 4 lanes) and through one
    launch per request on the same GPU, with identical results required."""
    import numpy as np
    import torch

    import paper_1701_01772_gb300 as gs
    import synth

    gs.build()
    base = synth.BASE_SEED + 4
    specs = [("er_2000", lambda s: synth.er(2000, 20000, s)),
             ("chung_lu_100k", lambda s: synth.chung_lu_100k(s)),
             ("chung_lu_1m", lambda s: synth.chung_lu(1_000_000, 20_000_000, 2.1, 50_000.0, s)),
             ("rmat_24", lambda s: synth.rmat(24, 16, s))]
    t0 = time.time()
    graphs, names = [], []
    for name, make in specs:
        for rep in range(2):
            graphs.append(make(base + 10 * len(graphs) + rep))
            names.append(name)
    gen_s = time.time() - t0
    all_bits = [3, 4, 7, 8, 9, 10, 11, 12]

    def draw(n_req, seed):
        rng = np.random.default_rng(seed)
        gidx = rng.integers(0, len(graphs), size=n_req)
        frac = 10 ** rng.uniform(-3, -1, size=n_req)
        seeds = rng.integers(1, 2**62, size=n_req)
        masks = []
        for i in range(n_req):
            bits = [b for b in all_bits if rng.random() < 0.5] or [3]
            if names[gidx[i]] == "rmat_24":
                bits = [b for b in bits if b in (3, 4)] or [3]
            masks.append(sum(1 << b for b in bits))
        return [(int(gidx[i]), float(frac[i]), int(seeds[i]), masks[i]) for i in range(n_req)]

    srv = gs.Server(hbm_budget_bytes=40 << 30, max_batch=64, lanes=4)
    ids = [srv.add_numpy(rp, col) for rp, col in graphs]
    t0 = time.time()
    srv.start(hub_budget_bytes=20 << 30)  # eight resident graphs share the GPU
    start_s = time.time() - t0
    singles = [gs.Graph.from_numpy(rp, col, hub_budget_bytes=20 << 30) for rp, col in graphs]
    for gi in range(len(graphs)):  # warm-up
        srv.wait(srv.submit(ids[gi], 0.001, 1, gs.GS_THREE_NODE))
        singles[gi].count_estimate(0.001, 1, gs.GS_THREE_NODE)
    torch.cuda.synchronize()

    def run_baseline(reqs, arrivals):
        """One launch per request, in arrival order, open loop."""
        lat, res = [], []
        t_begin = time.perf_counter()
        for (gi, f, sd, mk), at in zip(reqs, arrivals):
            delay = t_begin + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            r, _ = singles[gi].count_estimate(f, sd, mk)
            lat.append((time.perf_counter() - t_begin - at) * 1e3)
            res.append(r)
        return lat, res, time.perf_counter() - t_begin

    def run_server(reqs, arrivals):
        tickets = []
        t_begin = time.perf_counter()
        for (gi, f, sd, mk), at in zip(reqs, arrivals):
            delay = t_begin + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(ids[gi], f, sd, mk))
        lat, res = [], []
        for t in tickets:
            r, st = srv.wait(t, 900.0)
            lat.append(st["latency_s"] * 1e3)
            res.append(r)
        return lat, res, time.perf_counter() - t_begin

    def same(a_list, b_list):
        for ra, rb in zip(a_list, b_list):
            a, c = ra.as_dict(), rb.as_dict()
            for g in a:
                for key in ("X", "V"):
                    x, y = a[g][key], c[g][key]
                    if not ((x != x and y != y) or x == y):
                        return False
        return True

    # capacity of one launch per request: a burst run one by one
    n_cap = max(40, args.serve_requests // 2)
    cap_reqs = draw(n_cap, base + 1)
    lat, _, mk = run_baseline(cap_reqs, [0.0] * n_cap)
    capacity = n_cap / mk
    slat, _, smk = run_server(cap_reqs, [0.0] * n_cap)
    loads = [float(x) for x in args.serve_loads.split(",")]
    points = []
    for li, load in enumerate(loads + [None]):
        rate = args.serve_rate if load is None else load * capacity
        n_req = args.serve_requests
        reqs = draw(n_req, base + 10 + li)
        rng = np.random.default_rng(base + 100 + li)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req)).tolist()
        s_lat, s_res, s_mk = run_server(reqs, arrivals)
        b_lat, b_res, b_mk = run_baseline(reqs, arrivals)
        points.append({
            "offered": "spec 2000 req/s" if load is None else f"{load:.0%} of capacity",
            "rate_req_s": round(rate, 2), "requests": n_req,
            "server": {"p50_ms": round(percentile(s_lat, 50), 2),
                       "p99_ms": round(percentile(s_lat, 99), 2),
                       "req_s": round(n_req / s_mk, 2)},
            "one_launch_per_request": {"p50_ms": round(percentile(b_lat, 50), 2),
                                       "p99_ms": round(percentile(b_lat, 99), 2),
                                       "req_s": round(n_req / b_mk, 2)},
            "identical_results": same(s_res, b_res)})
    info = srv.info()
    srv.close()
    for g in singles:
        g.close()
    head = points[-1]
    return {
        "metric": "requests/s served (p50/p99 latency)", "value": head["server"]["req_s"],
        "unit": "req/s", "p50_ms": head["server"]["p50_ms"], "p99_ms": head["server"]["p99_ms"],
        "higher_is_better": True, "data": "synthetic",
        "config": {"workload": "serve: 8 resident graphs (ER 2000 x2, Chung-Lu 100k x2, Chung-Lu "
                               "1M x2, R-MAT 24 x2), Poisson arrivals, fractions log-uniform "
                               "[0.1%, 10%], random masks (3-node only on R-MAT)",
                   "budget_gb": 40, "lanes": 4, "generation_s": round(gen_s, 1),
                   "start_s": round(start_s, 2)},
        "capacity_one_launch_per_request_req_s": round(capacity, 2),
        "capacity_server_req_s": round(n_cap / smk, 2),
        "loads": points, "server": info,
    }


# ------------------------------------------------------------------ main

def line_from(r, args, world, steps, warmup, cpu=None):
    value = r["edges_all"] / (r["ms_total"] / 1e3)
    return {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup,
        "ms_per_step": round(r["ms_total"] / steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": r["desc"], "parts": r["parts"],
                   "l2": "flushed (256 MiB write) before every timed step; CSR > L2",
                   "hub_index": {k: r["graph"][k] for k in ("bitmap_hubs", "table_hubs")},
                   "parallelism": f"replicas x{world}"},
        "latency_ms": r["lat"], "part_stats_last_step": r["part_stats"],
        "graphlets_per_s": round(r["inc_all"] / (r["ms_total"] / 1e3), 1),
        "registration_s": r["registration_s"], "index_bytes": r["index_bytes"],
        "workspace_bytes": r["workspace_bytes"],
        "e2e": r["e2e"], "roofline": r["roofline"], "cpu_baseline": cpu,
        "gpu_launches": r["launches"], "clocks": r["clocks"],
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "batch":
        print(json.dumps(run_batch_bench(args)), flush=True)
        return
    if args.workload == "serve":
        print(json.dumps(run_serve_bench(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    name = args.workload
    rp, col = generate(name)
    r = run_gpu(args, rank, world, local, name, rp, col, args.steps, args.warmup)
    extra = None
    if name == "rmat_24" and not args.no_extra:
        rp2, col2 = generate("chung_lu_1m")
        es = max(1, min(args.steps, args.extra_steps))
        r2 = run_gpu(args, rank, world, local, "chung_lu_1m", rp2, col2, es, min(args.warmup, 3))
        extra = {"chung_lu_1m": line_from(r2, args, world, es, min(args.warmup, 3))}
        for key in ("metric", "unit", "n_gpus", "higher_is_better", "scaling", "vs_baseline",
                    "dtype", "data", "cpu_baseline", "e2e"):
            extra["chung_lu_1m"].pop(key, None)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            v, cores, sample, wall = oracle_step_rate(rp, col, WORKLOADS[name][1],
                                                      args.cpu_seconds)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{sample}; {wall:.1f} s wall on {cores} spawned processes (one "
                             "per core); per-edge rates scaled to the full step"}
        line = line_from(r, args, world, args.steps, args.warmup, cpu)
        if extra:
            line["extra"] = extra
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
