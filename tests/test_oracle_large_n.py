"""Oracle pins at large n: sparse graphs whose Step 3 sums pass 2^64.

The counts of a disjoint union of single edges, isolated nodes and a few small
components follow from the definition by binomial coefficients
(`disjoint_union.union_counts`).  That helper is itself pinned here against
brute-force enumeration on tiny unions; the oracle is then checked against it
on a graph of 2^27 nodes, where sum_e C(I,2) alone is about 2^66, so that an
oracle accumulating in 64 bits would fail.
"""
import numpy as np
import pytest

from disjoint_union import special_components, sparse_union_edges, union_counts
from oracle import bruteforce, oracle
from paper_1506_04322_gb300 import inputs


def _tiny_special():
    # triangle, path on three nodes, one K4 (11 nodes)
    return 11, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5),
                (6, 7), (6, 8), (6, 9), (7, 8), (7, 9), (8, 9)]


@pytest.mark.parametrize("n_iso,n_pairs,use_special", [
    (0, 0, True), (1, 0, True), (0, 2, False), (3, 2, False), (1, 2, False),
    (0, 1, True), (2, 1, True), (5, 3, False), (12, 0, False)])
def test_union_counts_match_bruteforce(n_iso, n_pairs, use_special):
    sn, sp = _tiny_special() if use_special else (0, [])
    if sn + 2 * n_pairs + n_iso > 13:
        sn, sp = 6, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5)]
    n = sn + 2 * n_pairs + n_iso
    edges = list(sp) + [(sn + 2 * i, sn + 2 * i + 1) for i in range(n_pairs)]
    g = inputs.from_edges(n, edges)
    assert union_counts(n_iso, n_pairs, sn, sp) == bruteforce.global_counts(g)


def test_union_counts_special_components_vs_bruteforce_parts():
    # the 33-node special set is too large to enumerate whole; each of its
    # components alone (plus two isolated nodes) is not
    sn, sp = special_components()
    comps, start = [], 0
    for size in (3, 4, 4, 5, 5, 4, 4, 4):
        comps.append((size, [(a - start, b - start) for a, b in sp if start <= a < start + size]))
        start += size
    assert start == sn
    for size, el in comps:
        g = inputs.from_edges(size + 2, el)
        assert union_counts(2, 0, size, el) == bruteforce.global_counts(g)


def test_oracle_exact_past_2_64():
    n = 1 << 27
    edges, n_iso = sparse_union_edges(n, 8192, 1 << 14)
    g = inputs.from_edges(n, edges)
    sn, sp = special_components()
    want = union_counts(n_iso, 8192, sn, sp)
    got, sums = oracle.alg2_global(g, with_sums=True)
    assert sums["nII"] > 1 << 64          # the case this pins
    assert got == want
    assert oracle.o2_global(g) == want
    # per-edge records of a few edges of each kind against the definition:
    # a lone edge (u, v) has I = n - 2 and lies in every 4-subset with one
    # other edge (g49) or none (g4_10)
    e = g.edges()
    m = e.shape[0]
    lone = oracle.edges_direct(g, e[:3])
    col = {x: i for i, x in enumerate(bruteforce.ORDER)}
    for row in lone:
        assert int(row[col["g33"]]) == n - 2
        assert int(row[col["g49"]]) == m - 1
        assert int(row[col["g4_10"]]) == (n - 2) * (n - 3) // 2 - (m - 1)
        assert all(int(row[col[x]]) == 0 for x in bruteforce.ORDER
                   if x not in ("g33", "g49", "g4_10"))
    assert np.array_equal(lone[0], lone[2])
