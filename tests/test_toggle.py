"""Local update on inserting or deleting one edge.

The brute-force toggle record (every subset holding both end nodes, typed
before and after) is pinned here against full recounts of the graph before
and after the toggle; the GPU's gains and losses must equal it exactly, and
on larger graphs their difference must equal the difference of two O2
recounts.
"""
import random

import numpy as np
import pytest

from oracle import bruteforce, oracle
from paper_1506_04322_gb300 import gd, inputs


def _toggled(g, u, v):
    e = {tuple(x) for x in g.edges().tolist()}
    key = (min(u, v), max(u, v))
    if key in e:
        e.remove(key)
    else:
        e.add(key)
    return inputs.from_edges(g.n, sorted(e))


def test_bruteforce_toggle_equals_recount_difference():
    rng = random.Random(11)
    for t in range(40):
        g = inputs.erdos_renyi(rng.randint(3, 10), rng.random(), 900 + t)
        u, v = rng.sample(range(g.n), 2)
        gain, loss = bruteforce.toggle_gain_loss(g, u, v)
        before = bruteforce.global_counts(g)
        after = bruteforce.global_counts(_toggled(g, u, v))
        assert [a - b for a, b in zip(after, before)] == [x - y for x, y in zip(gain, loss)]
        # every subset holding u and v changes type: n-2 triples, C(n-2, 2) quads
        assert sum(gain[:4]) == sum(loss[:4]) == g.n - 2
        assert sum(gain[4:]) == sum(loss[4:]) == (g.n - 2) * (g.n - 3) // 2


@pytest.mark.gpu
def test_toggle_matches_bruteforce():
    rng = random.Random(5)
    with gd.Context(0) as ctx:
        for t in range(60):
            g = inputs.erdos_renyi(rng.randint(3, 40), rng.random(), 1200 + t)
            e = g.edges()
            with ctx.graph(g) as h:
                pairs = [tuple(rng.sample(range(g.n), 2)) for _ in range(3)]
                if len(e):
                    pairs.append(tuple(int(x) for x in e[rng.randrange(len(e))]))
                for u, v in pairs:
                    gain, loss, was = h.toggle_delta(u, v)
                    bg, bl = bruteforce.toggle_gain_loss(g, u, v)
                    assert (gain, loss) == (bg, bl), (g.name, u, v)
                    assert was == (v in set(g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]))


@pytest.mark.gpu
def test_toggle_matches_recounts_on_larger_graphs():
    g = inputs.chung_lu(20_000, 2.2, 90_000, 0.0, 77)
    deg = g.degrees()
    e = g.edges()
    hubs = np.argsort(-deg)[:3]
    pairs = [(int(hubs[0]), int(hubs[1])), (int(hubs[0]), int(np.argmin(deg))), tuple(int(x) for x in e[0]),
             tuple(int(x) for x in e[len(e) // 2]), (1, 2)]
    before = oracle.o2_global(g)
    with gd.Context(0) as ctx, ctx.graph(g) as h:
        for u, v in pairs:
            if u == v:
                continue
            gain, loss, _ = h.toggle_delta(u, v)
            after = oracle.o2_global(_toggled(g, u, v))
            assert [a - b for a, b in zip(after, before)] == [x - y for x, y in zip(gain, loss)], (u, v)


@pytest.mark.gpu
def test_toggle_rejects_bad_pairs():
    g = inputs.erdos_renyi(30, 0.2, 3)
    with gd.Context(0) as ctx, ctx.graph(g) as h:
        for u, v in ((4, 4), (-1, 3), (3, 30)):
            with pytest.raises(gd.GDError) as ei:
                h.toggle_delta(u, v)
            assert ei.value.code == gd.GD_EINVAL
