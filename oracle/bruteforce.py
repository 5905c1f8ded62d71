"""O0: brute-force graphlet counts straight from the definitions (tiny graphs).

Test infrastructure only (see ``oracle.py``).

Definition (Sec. 2.1, Definitions 1-2 and the problem statement): the count of a
graphlet g of size k is the number of k-node subsets of V whose induced subgraph
is isomorphic to g.  Per edge e = (u, v): the number of such subsets that contain
both u and v.

Each induced subgraph is classified by the properties Table 1 lists for every
graphlet: its number of edges (density x C(k,2)), its maximum degree, its number
of triangles and its number of connected components.  These four values are
distinct for all 4 three-node and 11 four-node graphlets.

Pure Python; exponential in n, meant for n <= ~12.
"""
from __future__ import annotations

import itertools

# Table 1: graphlet -> (edges, max degree, triangles, components)
TABLE1_KEYS = {
    "g41": (6, 3, 4, 1), "g42": (5, 3, 2, 1), "g43": (4, 3, 1, 1), "g44": (4, 2, 0, 1),
    "g45": (3, 3, 0, 1), "g46": (3, 2, 0, 1), "g47": (3, 2, 1, 2), "g48": (2, 2, 0, 2),
    "g49": (2, 1, 0, 2), "g4_10": (1, 1, 0, 3), "g4_11": (0, 0, 0, 4),
    "g31": (3, 2, 1, 1), "g32": (2, 2, 0, 1), "g33": (1, 1, 0, 2), "g34": (0, 0, 0, 3),
}
ORDER = ["g31", "g32", "g33", "g34", "g41", "g42", "g43", "g44", "g45", "g46",
         "g47", "g48", "g49", "g4_10", "g4_11"]
_BY_KEY = {(k, key): name for name, key in TABLE1_KEYS.items()
           for k in [3 if name.startswith("g3") else 4]}


def adjacency_sets(g) -> list[set]:
    adj = [set() for _ in range(g.n)]
    for u in range(g.n):
        for p in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            adj[u].add(int(g.col_idx[p]))
    return adj


def classify(nodes, adj) -> str:
    """Graphlet name of the subgraph induced by `nodes` (3 or 4 nodes)."""
    nodes = list(nodes)
    k = len(nodes)
    deg = {x: 0 for x in nodes}
    edges = 0
    for a, b in itertools.combinations(nodes, 2):
        if b in adj[a]:
            edges += 1
            deg[a] += 1
            deg[b] += 1
    tri = sum(1 for a, b, c in itertools.combinations(nodes, 3)
              if b in adj[a] and c in adj[a] and c in adj[b])
    # components by union-find
    parent = {x: x for x in nodes}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in itertools.combinations(nodes, 2):
        if b in adj[a]:
            parent[find(a)] = find(b)
    comps = len({find(x) for x in nodes})
    return _BY_KEY[(k, (edges, max(deg.values()), tri, comps))]


def global_counts(g) -> list[int]:
    adj = adjacency_sets(g)
    cnt = dict.fromkeys(ORDER, 0)
    for k in (3, 4):
        for s in itertools.combinations(range(g.n), k):
            cnt[classify(s, adj)] += 1
    return [cnt[x] for x in ORDER]


def edge_counts(g, u: int, v: int) -> list[int]:
    """c_g(e) for e = (u, v): subsets containing both u and v."""
    adj = adjacency_sets(g) if not isinstance(g, list) else g
    n = len(adj)
    cnt = dict.fromkeys(ORDER, 0)
    others = [x for x in range(n) if x != u and x != v]
    for w in others:
        cnt[classify((u, v, w), adj)] += 1
    for w, r in itertools.combinations(others, 2):
        cnt[classify((u, v, w, r), adj)] += 1
    return [cnt[x] for x in ORDER]


def per_edge_counts(g) -> list[list[int]]:
    """Rows in CSR order of the undirected edges (u, v), u < v."""
    adj = adjacency_sets(g)
    rows = []
    for u in range(g.n):
        for p in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            v = int(g.col_idx[p])
            if v > u:
                rows.append(edge_counts(adj, u, v))
    return rows


def toggle_gain_loss(g, u: int, v: int) -> tuple[list[int], list[int]]:
    """For the pair {u, v} toggled (deleted if an edge, inserted if not): per
    graphlet, the number of 3- and 4-node subsets that enter it (gain) and
    leave it (loss).  Only subsets holding both u and v change; each is
    classified before and after from the definitions.  O(n^2) subsets."""
    adj = adjacency_sets(g)
    after = [set(s) for s in adj]
    if v in after[u]:
        after[u].discard(v); after[v].discard(u)
    else:
        after[u].add(v); after[v].add(u)
    gain = {name: 0 for name in ORDER}
    loss = {name: 0 for name in ORDER}
    others = [w for w in range(g.n) if w != u and w != v]
    subsets = [(u, v, w) for w in others]
    subsets += [(u, v, w, r) for w, r in itertools.combinations(others, 2)]
    for s in subsets:
        a, b = classify(s, adj), classify(s, after)
        if a != b:
            loss[a] += 1
            gain[b] += 1
    return [gain[x] for x in ORDER], [loss[x] for x in ORDER]
