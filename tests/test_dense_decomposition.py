"""Host check of how the 4-node pass splits the 4-clique count of a dense
edge (Alg. 3: k(e) = number of edges among T = N(u) cap N(v)).

For an edge whose T holds many hub-matrix vertices, the GPU counts, for
the dense slots s < D:
  - pairs of T members that both have a dense slot, by matrix rows ANDed
    with T's mask (each pair once, from the lower slot);
  - for every other member w: each matrix neighbour x of w (slot s) counts
    when s < D and x is in T, or when s >= D, x > w and x is in T; each
    neighbour x > w without a matrix slot counts when x is in T.
The sum must equal k(e) for every D, from 0 (no dense mode) to the whole
matrix. Plain Python sets, no GPU code."""
import itertools
import random

import pytest


def _graph(n, p, hubs, p_hub, seed):
    """Random graph with a few high-degree vertices (so T has matrix
    members and non-members)."""
    rng = random.Random(seed)
    adj = {v: set() for v in range(n)}
    for a, b in itertools.combinations(range(n), 2):
        q = p_hub if (a < hubs or b < hubs) else p
        if rng.random() < q:
            adj[a].add(b)
            adj[b].add(a)
    # relabel randomly so hubs are not the lowest ids
    perm = list(range(n))
    rng.shuffle(perm)
    return {perm[v]: {perm[x] for x in nb} for v, nb in adj.items()}


def _matrix_slots(adj, count):
    """Top `count` vertices by (degree, id) get slots in increasing id order
    (the registration's order)."""
    top = sorted(adj, key=lambda v: (-len(adj[v]), -v))[:count]
    return {v: s for s, v in enumerate(sorted(top))}


def _k_true(adj, u, v):
    T = adj[u] & adj[v]
    return sum(1 for a, b in itertools.combinations(sorted(T), 2) if b in adj[a])


def _k_split(adj, slot, D, u, v):
    T = adj[u] & adj[v]
    dense = {w for w in T if w in slot and slot[w] < D}
    k = 0
    # pairs of dense-slot members (matrix rows AND the mask, lower slot first)
    for w in dense:
        k += sum(1 for x in dense if slot[x] > slot[w] and x in adj[w])
    # the other members: matrix-neighbour list and non-matrix list above w
    for w in T - dense:
        for x in adj[w]:
            if x in slot:
                if slot[x] < D:
                    k += x in T
                else:
                    k += x > w and x in T
            elif x > w:
                k += x in T
    return k


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_split_equals_four_clique_count_for_every_dense_slot_limit(seed):
    adj = _graph(n=90, p=0.06, hubs=12, p_hub=0.7, seed=seed)
    slot = _matrix_slots(adj, 40)
    edges = [(u, v) for u in adj for v in adj[u] if u < v]
    rng = random.Random(seed)
    sample = rng.sample(edges, min(150, len(edges)))
    for D in (0, 8, 16, 32, 40, 128):
        for u, v in sample:
            assert _k_split(adj, slot, D, u, v) == _k_true(adj, u, v), (D, u, v)


def test_split_on_a_complete_graph_counts_every_pair_once():
    n = 30
    adj = {v: set(range(n)) - {v} for v in range(n)}
    slot = _matrix_slots(adj, 20)
    want = (n - 2) * (n - 3) // 2  # edges among the other n - 2 vertices
    for D in (0, 10, 20):
        assert _k_split(adj, slot, D, 0, 1) == want


def test_a_dropped_term_fails():
    """A plausible mistake in the split (the non-matrix neighbours of the
    other members left out) changes the count on these graphs."""
    adj = _graph(n=90, p=0.06, hubs=12, p_hub=0.7, seed=4)
    slot = _matrix_slots(adj, 40)

    def k_missing_nonmatrix(u, v):
        T = adj[u] & adj[v]
        dense = {w for w in T if slot.get(w, 1 << 30) < 32}
        k = sum(1 for w in dense for x in dense if slot[x] > slot[w] and x in adj[w])
        for w in T - dense:
            k += sum(1 for x in adj[w] if x in slot and ((slot[x] < 32 and x in T)
                                                        or (slot[x] >= 32 and x > w and x in T)))
        return k

    edges = [(u, v) for u in adj for v in adj[u] if u < v]
    assert any(k_missing_nonmatrix(u, v) != _k_true(adj, u, v) for u, v in edges)
