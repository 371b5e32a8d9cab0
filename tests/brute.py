"""Independent pins for the oracle: brute-force enumeration, Table 1
properties, closed forms and counting identities.  Pure Python / numpy; shares
nothing with the oracle's per-edge algorithm."""
from __future__ import annotations

import itertools
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Each graphlet of the paper's Table 1 written as (n, edge list).
GRAPHLET_EDGES = {
    3: (3, [(0, 1), (1, 2), (0, 2)]),                                   # triangle
    4: (3, [(0, 1), (1, 2)]),                                           # 2-star
    5: (3, [(0, 1)]),                                                   # 3-node-1-edge
    6: (3, []),                                                         # 3-node-independent
    7: (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),           # 4-clique
    8: (4, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)]),                   # chordal-cycle
    9: (4, [(0, 1), (0, 2), (1, 2), (0, 3)]),                           # tailed-triangle
    10: (4, [(0, 1), (1, 2), (2, 3), (3, 0)]),                          # 4-cycle
    11: (4, [(0, 1), (0, 2), (0, 3)]),                                  # 3-star
    12: (4, [(0, 1), (1, 2), (2, 3)]),                                  # 4-path
    13: (4, [(0, 1), (1, 2), (0, 2)]),                                  # 4-node-1-triangle
    14: (4, [(0, 1), (1, 2)]),                                          # 4-node-2-star
    15: (4, [(0, 1), (2, 3)]),                                          # 4-node-2-edge
    16: (4, [(0, 1)]),                                                  # 4-node-1-edge
    17: (4, []),                                                        # 4-node-independent
}


def load_table1() -> dict:
    rows = {}
    with open(os.path.join(GOLDEN, "table1_graphlets.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = {
                "n": int(p[1]), "rho": float(p[2]), "dmax": int(p[3]), "dbar": float(p[4]),
                "tri": int(p[5]), "core": int(p[6]), "chi": int(p[7]),
                "diam": math.inf if p[8] == "inf" else int(p[8]), "comp": int(p[9]),
            }
    return rows


def adjacency(n: int, edges) -> np.ndarray:
    A = np.zeros((n, n), dtype=np.int64)
    for a, b in edges:
        A[a, b] = A[b, a] = 1
    return A


def _components(A: np.ndarray) -> list:
    n = len(A)
    seen, comps = [False] * n, []
    for s in range(n):
        if seen[s]:
            continue
        stack, comp = [s], []
        seen[s] = True
        while stack:
            x = stack.pop()
            comp.append(x)
            for y in np.nonzero(A[x])[0]:
                if not seen[y]:
                    seen[y] = True
                    stack.append(int(y))
        comps.append(comp)
    return comps


def properties(n: int, edges) -> dict:
    """The Table 1 columns computed from an edge list."""
    A = adjacency(n, edges)
    deg = A.sum(1)
    m = len(edges)
    tri = int(np.trace(A @ A @ A) // 6)
    # degeneracy (max k-core number)
    alive, d, core = set(range(n)), deg.copy(), 0
    while alive:
        v = min(alive, key=lambda x: d[x])
        core = max(core, int(d[v]))
        alive.remove(v)
        for w in np.nonzero(A[v])[0]:
            if int(w) in alive:
                d[w] -= 1
    # chromatic number by trying k colours
    chi = 0
    for k in range(1, n + 1):
        if any(all(c[a] != c[b] for a, b in edges) for c in itertools.product(range(k), repeat=n)):
            chi = k
            break
    # diameter of the largest finite distances (BFS over all pairs)
    dist = np.full((n, n), np.inf)
    for s in range(n):
        dist[s, s] = 0
        frontier, k = [s], 0
        while frontier:
            k += 1
            nxt = []
            for x in frontier:
                for y in np.nonzero(A[x])[0]:
                    if dist[s, y] == np.inf:
                        dist[s, y] = k
                        nxt.append(int(y))
            frontier = nxt
    finite = dist[np.isfinite(dist) & (dist > 0)]
    diam = int(finite.max()) if finite.size else math.inf
    return {"n": n, "rho": 2 * m / (n * (n - 1)), "dmax": int(deg.max()), "dbar": 2 * m / n,
            "tri": tri, "core": core, "chi": chi, "diam": diam, "comp": len(_components(A))}


def classify4(A: np.ndarray, quad) -> int:
    """Graphlet id of the subgraph induced by 4 nodes, identified by the
    Table 1 triple (density, max degree, number of components)."""
    sub = A[np.ix_(quad, quad)]
    m = int(sub.sum()) // 2
    dmax = int(sub.sum(1).max())
    comp = len(_components(sub))
    table = {(6, 3, 1): 7, (5, 3, 1): 8, (4, 3, 1): 9, (4, 2, 1): 10, (3, 3, 1): 11,
             (3, 2, 1): 12, (3, 2, 2): 13, (2, 2, 2): 14, (2, 1, 2): 15, (1, 1, 3): 16,
             (0, 0, 4): 17}
    return table[(m, dmax, comp)]


def brute_counts(A: np.ndarray) -> dict:
    """Counts of every 3- and 4-node graphlet by enumerating node subsets."""
    n = len(A)
    out = {i: 0 for i in range(3, 18)}
    for tri in itertools.combinations(range(n), 3):
        m = int(A[np.ix_(tri, tri)].sum()) // 2
        out[{3: 3, 2: 4, 1: 5, 0: 6}[m]] += 1
    for quad in itertools.combinations(range(n), 4):
        out[classify4(A, quad)] += 1
    return out


def csr_from_adjacency(A: np.ndarray):
    n = len(A)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols = []
    for v in range(n):
        nb = np.nonzero(A[v])[0]
        cols.extend(int(x) for x in nb)
        row_ptr[v + 1] = len(cols)
    return row_ptr, np.asarray(cols, dtype=np.int32)


def csr_from_edges(n: int, edges):
    return csr_from_adjacency(adjacency(n, edges))


def adjacency_from_csr(row_ptr, col) -> np.ndarray:
    n = len(row_ptr) - 1
    A = np.zeros((n, n), dtype=np.int64)
    for v in range(n):
        A[v, col[row_ptr[v]:row_ptr[v + 1]]] = 1
    return A


# --------------------------------------------------------------- closed forms

def closed_form(kind: str, *args) -> dict:
    """Textbook counts of the connected graphlets for standard families."""
    c = math.comb
    z = {i: 0 for i in (3, 4, 7, 8, 9, 10, 11, 12)}
    if kind == "complete":
        (n,) = args
        z[3], z[7] = c(n, 3), c(n, 4)
    elif kind == "cycle":
        (n,) = args
        if n == 3:
            z[3] = 1
        elif n == 4:
            z[4], z[10] = 4, 1
        else:
            z[4], z[12] = n, n
    elif kind == "path":
        (n,) = args
        z[4], z[12] = max(n - 2, 0), max(n - 3, 0)
    elif kind == "star":
        (s,) = args
        z[4], z[11] = c(s, 2), c(s, 3)
    elif kind == "bipartite":
        a, b = args
        z[4] = a * c(b, 2) + b * c(a, 2)
        z[10] = c(a, 2) * c(b, 2)
        z[11] = a * c(b, 3) + b * c(a, 3)
    return z


def family_edges(kind: str, *args):
    if kind == "complete":
        (n,) = args
        return n, list(itertools.combinations(range(n), 2))
    if kind == "cycle":
        (n,) = args
        return n, [(i, (i + 1) % n) for i in range(n)]
    if kind == "path":
        (n,) = args
        return n, [(i, i + 1) for i in range(n - 1)]
    if kind == "star":
        (s,) = args
        return s + 1, [(0, i) for i in range(1, s + 1)]
    if kind == "bipartite":
        a, b = args
        return a + b, [(i, a + j) for i in range(a) for j in range(b)]
    raise ValueError(kind)


# --------------------------------------------------------------- identities

def identities(row_ptr, col) -> dict:
    """Degree- and walk-based quantities that fix linear combinations of the
    induced counts (non-induced subgraph counting):
      wedges   = sum_v C(d_v, 2)                     = G4 + 3 G3
      claws    = sum_v C(d_v, 3)                     = G11 + G9 + 2 G8 + 4 G7
      paths3   = sum_(u,v) (d_u-1)(d_v-1) - 3 G3     = G12 + 2 G9 + 4 G10 + 6 G8 + 12 G7
      cyc4     = (tr(A^4) - 2 sum d^2 + 2M) / 8      = G10 + G8 + 3 G7   (dense, small graphs)
    Returned as Python ints; ``paths3`` is returned before subtracting 3 G3."""
    d = np.diff(np.asarray(row_ptr)).astype(object)
    n = len(d)
    src = np.repeat(np.arange(n), np.diff(np.asarray(row_ptr)))
    col = np.asarray(col)
    up = src < col
    du = d[src[up]]
    dv = d[col[up]]
    out = {
        "wedges": int(sum(x * (x - 1) // 2 for x in d)),
        "claws": int(sum(x * (x - 1) * (x - 2) // 6 for x in d)),
        "paths3_raw": int(sum((a - 1) * (b - 1) for a, b in zip(du, dv))),
        "sum_d2": int(sum(x * x for x in d)),
        "M": int(up.sum()),
    }
    return out


def edge_roles(A: np.ndarray, u: int, v: int) -> dict:
    """Brute force over every 3- and 4-vertex set containing the edge (u, v):
    the induced subgraph's graphlet and the edge's role in it.

    Keys: 'tri' (triangles with e), 'wedge' (2-stars with e), 'lone'
    (3-sets where e is the only edge), 'k4', 'diamond_chord' (e joins the
    two degree-3 vertices), 'diamond_rim', 'tailed_tail' (e is the pendant
    edge of a tailed triangle), 'tailed_other', 'c4', 'star' (3-stars with
    e), 'path_mid' (e is the middle edge of a 4-path), 'path_end',
    'tri_far' (pairs w in T, r adjacent to neither u nor v)."""
    n = len(A)
    others = [x for x in range(n) if x not in (u, v)]
    out = {k: 0 for k in ("tri", "wedge", "lone", "k4", "diamond_chord", "diamond_rim",
                          "tailed_tail", "tailed_other", "c4", "star", "path_mid", "path_end",
                          "tri_far")}
    for w in others:
        e = A[u, w] + A[v, w]
        out["tri" if e == 2 else "wedge" if e == 1 else "lone"] += 1
    for w, r in itertools.combinations(others, 2):
        S = [u, v, w, r]
        sub = A[np.ix_(S, S)]
        deg = sub.sum(1)
        m = int(sub.sum()) // 2
        du, dv = int(deg[0]), int(deg[1])
        if m == 6:
            out["k4"] += 1
        elif m == 5:
            out["diamond_chord" if du == 3 and dv == 3 else "diamond_rim"] += 1
        elif m == 4:
            if sorted(deg.tolist()) == [2, 2, 2, 2]:
                out["c4"] += 1
            else:
                out["tailed_tail" if min(du, dv) == 1 else "tailed_other"] += 1
        elif m == 3:
            s = sorted(deg.tolist())
            if s == [1, 1, 1, 3]:
                out["star"] += 1
            elif s == [1, 1, 2, 2]:
                out["path_mid" if du == 2 and dv == 2 else "path_end"] += 1
        for a_, b_ in ((w, r), (r, w)):
            if A[u, a_] and A[v, a_] and not A[u, b_] and not A[v, b_]:
                out["tri_far"] += 1
    return out
