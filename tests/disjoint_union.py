"""Exact graphlet counts of a sparse disjoint union, from the definition.

The graph is: `n_isolated` isolated nodes, `n_pairs` components that are a
single edge, and one small graph `special` (a list of edges on the nodes
0..special_n-1; it may itself hold several components).  By the problem
statement of Sec. 2.1, the count of a k-node graphlet is the number of
k-subsets whose induced subgraph is isomorphic to it.  A k-subset takes a set
S of the special nodes, b whole single-edge components, and r further nodes
that are isolated inside the subset (a single node of a single-edge component,
or an isolated node).  Its induced subgraph is G[S] plus b disjoint edges plus
r isolated nodes, classified by Table 1's keys; binomial coefficients count
the choices among the identical components.  Python integers: exact at any n.

Test helper only; independent of the oracle's and the library's arithmetic.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np

from oracle import bruteforce


def union_counts(n_isolated: int, n_pairs: int, special_n: int, special_edges) -> list[int]:
    adj_s = [set() for _ in range(special_n)]
    for a, b in special_edges:
        adj_s[a].add(b)
        adj_s[b].add(a)
    cnt = dict.fromkeys(bruteforce.ORDER, 0)
    for k in (3, 4):
        for s in range(0, min(k, special_n) + 1):
            for S in itertools.combinations(range(special_n), s):
                for b in range(0, (k - s) // 2 + 1):
                    r = k - s - 2 * b
                    # a of the r lone nodes come from distinct single-edge
                    # components (2 ways each), r - a from isolated nodes; the
                    # b whole components are chosen among the rest
                    ways = sum(comb(n_isolated, r - a) * comb(n_pairs, a) * 2 ** a * comb(n_pairs - a, b)
                               for a in range(min(r, n_pairs) + 1))
                    if ways == 0:
                        continue
                    adj = [set() for _ in range(k)]
                    for i, x in enumerate(S):
                        for j, y in enumerate(S):
                            if y in adj_s[x]:
                                adj[i].add(j)
                    for t in range(b):
                        p, q = s + 2 * t, s + 2 * t + 1
                        adj[p].add(q)
                        adj[q].add(p)
                    cnt[bruteforce.classify(range(k), adj)] += ways
    return [cnt[x] for x in bruteforce.ORDER]


# a few small components with every kind of edge: triangle, 4-cycle, K4, K5,
# star K_{1,4}, path P4, tailed triangle, diamond (33 nodes)
def special_components() -> tuple[int, list[tuple[int, int]]]:
    edges: list[tuple[int, int]] = []
    base = 0

    def add(k, el):
        nonlocal base
        edges.extend((base + a, base + b) for a, b in el)
        base += k

    add(3, [(0, 1), (1, 2), (0, 2)])
    add(4, [(0, 1), (1, 2), (2, 3), (0, 3)])
    add(4, [(a, b) for a in range(4) for b in range(a + 1, 4)])
    add(5, [(a, b) for a in range(5) for b in range(a + 1, 5)])
    add(5, [(0, i) for i in range(1, 5)])
    add(4, [(0, 1), (1, 2), (2, 3)])
    add(4, [(0, 1), (1, 2), (0, 2), (2, 3)])
    add(4, [(0, 1), (1, 2), (2, 3), (0, 3), (0, 2)])
    return base, edges


def sparse_union_edges(n: int, n_pairs: int, stride: int):
    """Edges of the union on n nodes as an (m, 2) int32 array: pair i is
    (stride*i, stride*i + 1); the special components sit on the top ids.
    Returns (edges, n_isolated)."""
    special_n, sp = special_components()
    top = n - special_n
    assert stride >= 2 and (n_pairs == 0 or stride * (n_pairs - 1) + 1 < top)
    first = np.arange(n_pairs, dtype=np.int64) * stride
    pairs = np.stack([first, first + 1], axis=1)
    spec = np.array(sp, dtype=np.int64) + top
    edges = np.concatenate([pairs, spec]).astype(np.int32)
    return edges, n - 2 * n_pairs - special_n
