"""Pins for the CPU oracle: everything here checks the oracle against something
other than itself -- worked examples, a library isomorphism test, closed forms,
the complement relation, brute force on tiny graphs, invariants, and planted
mistakes that the pins must catch."""
import itertools
import math
import os
import random

import numpy as np
import pytest

from oracle import bruteforce, oracle
from paper_1506_04322_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ORDER = bruteforce.ORDER
# edges of each graphlet (Table 1), used by the sum invariant
EDGES_OF = [3, 2, 1, 0, 6, 5, 4, 4, 3, 3, 3, 2, 2, 1, 0]


def load_graphlets():
    rows = []
    with open(os.path.join(GOLDEN, "graphlets.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip() if line.startswith("#") else line.strip()
            if not line:
                continue
            parts = line.split()
            name, k, desc, edges, comp = parts[:5]
            census = [int(x) for x in parts[5:9]]
            el = [] if edges == "-" else [(int(e[0]), int(e[1])) for e in edges.split(",")]
            rows.append(dict(name=name, k=int(k), desc=desc, edges=el, comp=comp, census=census))
    return rows


GRAPHLETS = load_graphlets()


def complement(g):
    adj = bruteforce.adjacency_sets(g)
    el = [(a, b) for a, b in itertools.combinations(range(g.n), 2) if b not in adj[a]]
    return inputs.from_edges(g.n, el)


def random_graphs(count, nmax, seed):
    rng = random.Random(seed)
    out = []
    for t in range(count):
        n = rng.randint(0, nmax)
        p = rng.random()
        out.append(inputs.erdos_renyi(n, p, 1000 * seed + t))
    return out


# --------------------------------------------------------------------------
# the brute force itself
# --------------------------------------------------------------------------

def test_bruteforce_classifier_matches_isomorphism():
    """Table 1 keys (edges, max degree, triangles, components) classify every
    labelled graph on 3 and 4 nodes exactly as graph isomorphism does."""
    nx = pytest.importorskip("networkx")
    refs = {}
    for r in GRAPHLETS:
        h = nx.Graph()
        h.add_nodes_from(range(r["k"]))
        h.add_edges_from(r["edges"])
        refs[r["name"]] = h
    for k in (3, 4):
        pairs = list(itertools.combinations(range(k), 2))
        seen = set()
        for mask in range(1 << len(pairs)):
            el = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            g = inputs.from_edges(k, el)
            name = bruteforce.classify(range(k), bruteforce.adjacency_sets(g))
            h = nx.Graph()
            h.add_nodes_from(range(k))
            h.add_edges_from(el)
            iso = [nm for nm, ref in refs.items() if ref.number_of_nodes() == k
                   and nx.is_isomorphic(h, ref)]
            assert iso == [name]
            seen.add(name)
        assert len(seen) == (4 if k == 3 else 11)


@pytest.mark.parametrize("row", GRAPHLETS, ids=lambda r: r["name"])
def test_worked_example_single_graphlet(row):
    """A graph that is itself graphlet g contains exactly one g (Table 1)."""
    g = inputs.from_edges(row["k"], row["edges"])
    want = [0] * 15
    if row["k"] == 4:
        want[:4] = row["census"]
    want[ORDER.index(row["name"])] += 1
    assert bruteforce.global_counts(g) == want
    assert oracle.alg2_global(g) == want
    assert oracle.o2_global(g, threads=1) == want


# --------------------------------------------------------------------------
# O1 (literal Algorithm 2) and O2 against brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_global_vs_bruteforce(seed):
    for g in random_graphs(60, 11, seed):
        bf = bruteforce.global_counts(g)
        assert oracle.alg2_global(g) == bf
        assert oracle.o2_global(g, threads=2) == bf
        assert oracle.triad_census(g) == bf[:4]


@pytest.mark.parametrize("seed", [4, 5])
def test_per_edge_vs_bruteforce(seed):
    for g in random_graphs(40, 10, seed):
        bf = np.array(bruteforce.per_edge_counts(g), dtype=np.uint64).reshape(-1, 15)
        assert np.array_equal(oracle.alg2_per_edge(g), bf)
        assert np.array_equal(oracle.o2_per_edge(g, threads=2), bf)
        e = g.edges()
        if len(e):
            sel = e[::-1]  # reversed orientation and order
            assert np.array_equal(oracle.edges_direct(g, sel[:, ::-1]), bf[::-1])


def test_structured_graphs_vs_bruteforce():
    """Skewed/structured tiny graphs (stars with chords, BA, dense) too."""
    graphs = [inputs.barabasi_albert(11, m, s) for m in (1, 2, 3) for s in range(4)]
    graphs += [inputs.erdos_renyi(9, 0.9, s) for s in range(4)]
    for g in graphs:
        bf = bruteforce.global_counts(g)
        assert oracle.alg2_global(g) == bf
        assert oracle.o2_global(g, threads=2) == bf
        pe = np.array(bruteforce.per_edge_counts(g), dtype=np.uint64).reshape(-1, 15)
        assert np.array_equal(oracle.o2_per_edge(g), pe)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

C = math.comb


def closed_complete(n):
    f = [0] * 15
    f[0] = C(n, 3)
    f[4] = C(n, 4)
    return f


def closed_star(k):                     # K_{1,k}: n = k+1
    f = [0] * 15
    f[1] = C(k, 2)
    f[3] = C(k, 3)
    f[8] = C(k, 3)
    f[14] = C(k, 4)
    return f


def closed_bipartite(a, b):
    f = [0] * 15
    f[1] = a * C(b, 2) + b * C(a, 2)
    f[3] = C(a, 3) + C(b, 3)
    f[7] = C(a, 2) * C(b, 2)
    f[8] = C(a, 3) * b + C(b, 3) * a
    f[14] = C(a, 4) + C(b, 4)
    return f


def closed_cycle(n):                    # C_n, n >= 6
    f = [0] * 15
    f[1] = n
    f[2] = n * (n - 4)
    f[3] = C(n, 3) - n - n * (n - 4)
    f[9] = n
    f[11] = n * (n - 5)
    f[12] = n * (n - 5) // 2
    f[13] = n * (C(n - 4, 2) - (n - 5))
    f[14] = C(n, 4) - sum(f[4:14])
    return f


def closed_empty(n):
    f = [0] * 15
    f[3] = C(n, 3)
    f[14] = C(n, 4)
    return f


def K(n):
    return inputs.from_edges(n, list(itertools.combinations(range(n), 2)))


CLOSED = (
    [(f"K{n}", lambda n=n: K(n), lambda n=n: closed_complete(n)) for n in (4, 5, 9, 40)]
    + [(f"star{k}", lambda k=k: inputs.from_edges(k + 1, [(0, i) for i in range(1, k + 1)]),
        lambda k=k: closed_star(k)) for k in (3, 7, 200)]
    + [(f"K{a},{b}", lambda a=a, b=b: inputs.from_edges(
        a + b, [(i, a + j) for i in range(a) for j in range(b)]),
        lambda a=a, b=b: closed_bipartite(a, b)) for a, b in ((2, 3), (4, 4), (7, 30))]
    + [(f"C{n}", lambda n=n: inputs.from_edges(n, [(i, (i + 1) % n) for i in range(n)]),
        lambda n=n: closed_cycle(n)) for n in (6, 7, 12, 101)]
    + [(f"empty{n}", lambda n=n: inputs.from_edges(n, []), lambda n=n: closed_empty(n))
       for n in (0, 1, 3, 50)]
)


@pytest.mark.parametrize("name,make,want", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(name, make, want):
    g = make()
    w = want()
    assert oracle.alg2_global(g) == w
    assert oracle.o2_global(g, threads=2) == w
    if g.n <= 12:
        assert bruteforce.global_counts(g) == w


# --------------------------------------------------------------------------
# complement relation (Sec. 2.2): f(g, G) = f(g_bar, G_bar)
# --------------------------------------------------------------------------

def test_complement_relation():
    comp = {r["name"]: r["comp"] for r in GRAPHLETS}
    for g in random_graphs(25, 12, 9) + [inputs.erdos_renyi(60, 0.3, 77)]:
        f = oracle.alg2_global(g)
        fb = oracle.o2_global(complement(g), threads=2)
        for i, name in enumerate(ORDER):
            assert f[i] == fb[ORDER.index(comp[name])], name


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def test_per_edge_sums_to_global_and_subsets():
    for g in random_graphs(10, 40, 11) + [inputs.erdos_renyi(300, 0.05, 3),
                                          inputs.barabasi_albert(300, 3, 5)]:
        f = oracle.alg2_global(g)
        pe = oracle.alg2_per_edge(g)
        assert np.array_equal(pe, oracle.o2_per_edge(g, threads=3))
        col = [int(x) for x in pe.astype(object).sum(axis=0)] if len(pe) else [0] * 15
        for i in range(15):
            assert col[i] == EDGES_OF[i] * f[i]
        assert sum(f[:4]) == C(g.n, 3)
        assert sum(f[4:]) == C(g.n, 4)


def test_sums_divisibility():
    g = inputs.erdos_renyi(400, 0.04, 12)
    _, s = oracle.alg2_global(g, with_sums=True)
    assert s["sT"] % 3 == 0 and s["sS"] % 2 == 0
    assert s["sCliq"] % 6 == 0 and s["sCyc"] % 4 == 0


def test_o1_and_o2_agree_on_first_workload():
    g = inputs.erdos_renyi_small()
    a, sa = oracle.alg2_global(g, with_sums=True)
    b, sb = oracle.o2_global(g, with_sums=True)
    assert a == b and sa == sb
    assert np.array_equal(oracle.alg2_per_edge(g), oracle.o2_per_edge(g))


def test_per_edge_is_local():
    """A per-edge record depends on the edge alone: sampled edges equal rows."""
    g = inputs.barabasi_albert(2000, 4, 21)
    full = oracle.o2_per_edge(g)
    e = g.edges()
    idx = np.random.default_rng(0).choice(len(e), 300, replace=False)
    assert np.array_equal(oracle.edges_direct(g, e[idx]), full[idx])


# --------------------------------------------------------------------------
# planted mistakes: the pins above must notice a dropped term or wrong sign
# --------------------------------------------------------------------------

@pytest.mark.parametrize("field,delta", [("nTT", -6), ("nSuSv", 4), ("nTS", 2), ("nSS", -3),
                                         ("nTI", 3), ("nSI", -2), ("nII", 1), ("nII1", 2),
                                         ("sCliq", 6), ("sCyc", -4), ("sI", 1)])
def test_planted_sum_error_is_caught(field, delta):
    g = inputs.erdos_renyi(11, 0.5, 3)
    bf = bruteforce.global_counts(g)
    f, s = oracle.alg2_global(g, with_sums=True)
    assert f == bf
    bad = dict(s)
    bad[field] = s[field] + delta
    try:
        got = oracle.complete(bad, g.n)
    except oracle.OracleError:
        return          # caught by exact-division / underflow checks
    assert got != bf


def test_inexact_division_is_an_error():
    g = inputs.erdos_renyi(11, 0.5, 3)
    _, s = oracle.alg2_global(g, with_sums=True)
    bad = dict(s)
    bad["sT"] += 1
    with pytest.raises(oracle.OracleError):
        oracle.complete(bad, g.n)


def test_invalid_csr_rejected():
    g = inputs.erdos_renyi(20, 0.3, 2)
    bad = inputs.Graph(g.n, g.row_ptr.copy(), g.col_idx.copy())
    if bad.nnz >= 2:
        r0 = int(bad.row_ptr[0]), int(bad.row_ptr[1])
        bad.col_idx[r0[0]] = 0   # self-loop on node 0 (or disorder)
        with pytest.raises(oracle.OracleError):
            oracle.alg2_global(bad)
