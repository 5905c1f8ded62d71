"""Ranking by graphlet counts and graphlet frequency features.

gd_gfd rounds each exact rational count / C(n, k) once to the nearest double;
Python's int / int true division is correctly rounded, so it is the
reference for the rounding.  Top-k ranking is compared with a numpy sort by
(value descending, index ascending), which makes the answer unique.
"""
import math
import random

import numpy as np
import pytest

from oracle import bruteforce, oracle
from paper_1506_04322_gb300 import gd, inputs


def _expected_gfd(n, m, counts):
    c2, c3, c4 = math.comb(n, 2), math.comb(n, 3), math.comb(n, 4)
    out = [m / c2 if c2 else 0.0, (c2 - m) / c2 if c2 else 0.0]
    out += [c / c3 if c3 else 0.0 for c in counts[:4]]
    out += [c / c4 if c4 else 0.0 for c in counts[4:]]
    return out


def test_gfd_rounding_random_rationals():
    """Random numerators below C(n, k) for n up to 2^31: bit-equal to the
    correctly rounded quotient."""
    rng = random.Random(7)
    for _ in range(400):
        n = rng.choice([rng.randint(4, 60), rng.randint(100, 10**6), rng.randint(10**8, 2**31 - 1)])
        m = rng.randint(0, math.comb(n, 2))
        counts = [rng.randint(0, math.comb(n, 3)) for _ in range(4)] + \
                 [rng.randint(0, math.comb(n, 4)) for _ in range(11)]
        got = gd.gd_gfd(n, m, counts)
        want = _expected_gfd(n, m, counts)
        assert [float(x) for x in got] == want


def test_gfd_rounding_ties_and_edges():
    """Numerators at the ends of the range and quotients with long binary
    expansions; 0 and 1 are exact."""
    n = 2**31 - 1
    c4 = math.comb(n, 4)
    # numerators that put the quotient exactly between two doubles
    for num in (c4 // 2, c4 // 3, 1, c4 - 1, c4):
        counts = [0] * 4 + [num] + [0] * 10
        assert float(gd.gd_gfd(n, 0, counts)[6]) == num / c4
    # an exact tie needs a power-of-two denominator, which C(n, k) is not for
    # k >= 2 and n > k: quotients with long binary expansions instead
    n = 1_000_003
    c3 = math.comb(n, 3)
    for num in range(1, 2000, 37):
        counts = [num * 12345 % c3, 0, 0, 0] + [0] * 11
        assert float(gd.gd_gfd(n, 5, counts)[2]) == counts[0] / c3


def test_gfd_closed_forms():
    """K_n: every 3- and 4-subset is a clique; the empty graph: none; a
    graph with fewer than k nodes has no k-subsets (0)."""
    for n in (4, 7, 12):
        g = inputs.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
        f = gd.gd_gfd(n, g.m, bruteforce.global_counts(g))
        assert f[0] == 1.0 and f[1] == 0.0 and f[2] == 1.0 and f[6] == 1.0
        assert sum(f[3:6]) == 0.0 and sum(f[7:]) == 0.0
    f = gd.gd_gfd(9, 0, bruteforce.global_counts(inputs.from_edges(9, [])))
    assert f[1] == 1.0 and f[5] == 1.0 and f[16] == 1.0
    assert list(gd.gd_gfd(3, 3, [1] + [0] * 14)[6:]) == [0.0] * 11
    with pytest.raises(gd.GDError):
        gd.gd_gfd(4, 7, [0] * 15)           # more edges than pairs


def _topk_ref(vals, k):
    # exact order for uint64 values: (value descending, index ascending)
    order = sorted(range(len(vals)), key=lambda i: (-int(vals[i]), i))[:k]
    return np.array(order, dtype=np.int64)


@pytest.mark.gpu
def test_topk_matches_sort():
    torch = pytest.importorskip("torch")
    g = inputs.chung_lu(20_000, 2.3, 90_000, 0.0, 21)
    pe = oracle.o2_per_edge(g)
    with gd.Context(0) as ctx:
        for col in (0, 1, 4, 7, 9, 3):           # column 3 is all zeros: every entry ties
            vals = np.ascontiguousarray(pe[:, col])
            for k in (0, 1, 17, 1000, len(vals)):
                want = _topk_ref(vals, k)
                idx, v = ctx.topk(pe, k, column=col)
                assert np.array_equal(idx, want), (col, k)
                assert np.array_equal(v, vals[want])
            dev = torch.from_numpy(pe.view(np.int64)).cuda()
            idx, _ = ctx.topk(dev, 250, column=col)
            assert np.array_equal(idx, _topk_ref(vals, 250))
        # a plain vector with many equal values
        rng = np.random.default_rng(3)
        x = rng.integers(0, 40, size=100_003).astype(np.uint64)
        x[::7] = np.uint64(2**64 - 1)
        idx, v = ctx.topk(x, 5000)
        assert np.array_equal(idx, _topk_ref(x, 5000))


@pytest.mark.gpu
def test_node_sums_and_node_triangles():
    g = inputs.barabasi_albert(3000, 4, 2)
    with gd.Context(0) as ctx, ctx.graph(g) as h:
        pe, _ = h.count_per_edge()
        e = g.edges()
        for col in (0, 4, 9):
            want = np.zeros(g.n, dtype=np.uint64)
            np.add.at(want, e[:, 0], pe[:, col])
            np.add.at(want, e[:, 1], pe[:, col])
            assert np.array_equal(h.node_sums(pe, col), want)
        # triangles at each node, from the definition, on a small graph
    small = inputs.erdos_renyi(40, 0.3, 5)
    with gd.Context(0) as ctx, ctx.graph(small) as h:
        pe, _ = h.count_per_edge()
        tri = h.node_sums(pe, 0)
        adj = [set(small.col_idx[small.row_ptr[v]:small.row_ptr[v + 1]]) for v in range(small.n)]
        for v in range(small.n):
            t = sum(1 for a in adj[v] for b in adj[v] if a < b and b in adj[a])
            assert int(tri[v]) == 2 * t


@pytest.mark.gpu
def test_gfd_batch_matches_exact_division():
    torch = pytest.importorskip("torch")
    graphs = inputs.graph_batch(300, seed=4)
    pk = inputs.pack(graphs)
    with gd.Context(0) as ctx:
        counts = ctx.count_batch(pk)
        d_np = torch.from_numpy(pk.graph_node_ptr).cuda()
        d_rp = torch.from_numpy(pk.row_ptr).cuda()
        d_c = torch.from_numpy(np.ascontiguousarray(counts).view(np.int64)).cuda()
        out = torch.zeros((len(graphs), 17), dtype=torch.float64, device="cuda")
        gd.gd_gfd_batch(ctx.handle, len(graphs), d_np.data_ptr(), d_rp.data_ptr(), d_c.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    for i, gg in enumerate(graphs):
        want = _expected_gfd(gg.n, gg.m, [int(x) for x in counts[i]])
        assert [float(x) for x in got[i]] == want, i
