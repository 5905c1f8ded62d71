"""GPU parity on a sparse graph of 2^28 nodes: the Step 3 sums pass 2^64.

2^20 single-edge components spread over the whole id range, a few small
components on the top ids, every other node isolated.  Per edge, C(I,2) is
about 2^55, so sum_e C(I,2) is about 2^75, and every CTA's partial of it
passes 2^64: the library must keep them in 128 bits (Lemma 7, Eq. g4_11).
Checked against counts from the definition in Python integers, against the
literal Algorithm 2 oracle, and per edge against the subset-count invariant
and the oracle's per-edge records.
"""
import numpy as np
import pytest

from disjoint_union import special_components, sparse_union_edges, union_counts
from oracle import bruteforce, oracle
from paper_1506_04322_gb300 import gd, inputs

pytestmark = pytest.mark.gpu

EDGES_OF = [3, 2, 1, 0, 6, 5, 4, 4, 3, 3, 3, 2, 2, 1, 0]   # |E(g)|, Table 1 order


def test_sparse_graph_of_2_28_nodes():
    n, pairs = 1 << 28, 1 << 20
    edges, n_iso = sparse_union_edges(n, pairs, 256)
    g = inputs.from_edges(n, edges)
    sn, sp = special_components()
    want = union_counts(n_iso, pairs, sn, sp)
    with gd.Context(0) as ctx, ctx.graph(g, validate=True) as h:
        glob = h.count_global()
        pe, glob2 = h.count_per_edge()
    assert glob == want
    assert glob2 == want
    assert oracle.alg2_global(g) == want
    # sum_e c_g(e) = |E(g)| f(g), in Python integers
    for c in range(15):
        assert int(pe[:, c].astype(object).sum()) == EDGES_OF[c] * want[c], bruteforce.ORDER[c]
    # per-edge records: every edge of the small components, and lone edges
    # from the whole id range
    e = g.edges()
    rng = np.random.default_rng(7)
    idx = np.concatenate([np.arange(pairs, e.shape[0]), rng.choice(pairs, 64, replace=False)])
    assert np.array_equal(pe[idx], oracle.edges_direct(g, e[idx]))
