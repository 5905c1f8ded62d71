"""GPU parity: libgd (CUDA, through the C ABI) against the CPU oracle.

All counts are exact integers, so the bar is bit-exact equality of every global
count and every per-edge column.
"""
import hashlib
import json
import os
import random

import numpy as np
import pytest

from oracle import bruteforce, oracle
from paper_1506_04322_gb300 import gd, inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "workloads.json")
VARIANTS = [gd.GD_VARIANT_ORIENTED, gd.GD_VARIANT_LITERAL]


@pytest.fixture(scope="module")
def ctxs():
    out = {v: gd.Context(0, variant=v) for v in VARIANTS}
    # a context whose shared-memory wedge table is tiny, so the global-table
    # tier of the 4-cycle kernel runs on small graphs too
    out["tiny_table"] = gd.Context(0, variant=gd.GD_VARIANT_ORIENTED, smem_table_max=256)
    # every scheduling tier on small graphs: hub batches from max(2^6, n/8) wedges, and
    # the global-scratch 4-clique kernel for out-degrees above 8
    out["all_tiers"] = gd.Context(0, variant=gd.GD_VARIANT_ORIENTED, smem_table_max=256,
                                  bitmap_max_outdeg=8, hub_wedges_log2=6)
    # global counts of every hub by per-node hub masks (pull form), or of none
    out["pull_always"] = gd.Context(0, variant=gd.GD_VARIANT_ORIENTED, smem_table_max=256,
                                    hub_wedges_log2=6, hub_pull=gd.GD_PULL_ALWAYS)
    out["pull_never"] = gd.Context(0, variant=gd.GD_VARIANT_ORIENTED, smem_table_max=256,
                                   hub_wedges_log2=6, hub_pull=gd.GD_PULL_NEVER)
    yield out
    for c in out.values():
        c.close()


def run_both(ctx, g):
    with ctx.graph(g) as h:
        glob = h.count_global()
        pe, glob2 = h.count_per_edge()
    assert glob == glob2
    return glob, pe


def random_graphs(count, nmax, seed):
    rng = random.Random(seed)
    return [inputs.erdos_renyi(rng.randint(0, nmax), rng.random(), 7000 * seed + t) for t in range(count)]


def structured_graphs():
    gs = []
    for n in (1, 2, 3, 4, 5, 33):
        gs.append(inputs.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)]))
    for k in (1, 31, 32, 33, 700, 5000):
        gs.append(inputs.from_edges(k + 1, [(0, i) for i in range(1, k + 1)]))
    for a, b in ((2, 3), (5, 40), (33, 65)):
        gs.append(inputs.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)]))
    for n in (6, 97):
        gs.append(inputs.from_edges(n, [(i, (i + 1) % n) for i in range(n)]))
    gs.append(inputs.from_edges(0, []))
    gs.append(inputs.from_edges(17, []))
    # hub attached to a dense core: exercises every scheduling tier
    el = [(0, i) for i in range(1, 6001)] + [(i, i + 1) for i in range(1, 6000)]
    el += [(i, j) for i in range(1, 60) for j in range(i + 2, 60)]
    gs.append(inputs.from_edges(6001, el))
    gs += [inputs.barabasi_albert(3000, m, 5 + m) for m in (1, 3, 8)]
    return gs


ALL_CTX = VARIANTS + ["tiny_table", "all_tiers", "pull_always", "pull_never"]


@pytest.mark.parametrize("variant", ALL_CTX)
def test_tiny_graphs_match_bruteforce(ctxs, variant):
    for g in random_graphs(80, 11, 1):
        glob, pe = run_both(ctxs[variant], g)
        assert glob == bruteforce.global_counts(g)
        bf = np.array(bruteforce.per_edge_counts(g), dtype=np.uint64).reshape(-1, 15)
        assert np.array_equal(pe, bf)


@pytest.mark.parametrize("variant", ALL_CTX)
def test_structured_graphs_match_oracle(ctxs, variant):
    for g in structured_graphs():
        glob, pe = run_both(ctxs[variant], g)
        assert glob == oracle.o2_global(g), g.name
        assert np.array_equal(pe, oracle.o2_per_edge(g)), g.name


@pytest.mark.parametrize("variant", ALL_CTX)
def test_medium_random_graphs(ctxs, variant):
    gs = [inputs.erdos_renyi(n, p, s) for s, (n, p) in enumerate([(257, 0.3), (1000, 0.02), (4099, 0.003)])]
    gs += [inputs.chung_lu(20_000, 2.2, 90_000, 0.0, 3), inputs.chung_lu(200_000, 2.05, 900_000, 0.0, 6)]
    for g in gs:
        glob, pe = run_both(ctxs[variant], g)
        assert glob == oracle.o2_global(g), g.name
        assert np.array_equal(pe, oracle.o2_per_edge(g)), g.name


@pytest.mark.parametrize("variant", VARIANTS)
def test_erdos_renyi_workload_full(ctxs, variant):
    """G(2000, 0.005): every global count and every per-edge column vs the
    literal Algorithm 2 oracle."""
    g = inputs.erdos_renyi_small()
    glob, pe = run_both(ctxs[variant], g)
    assert glob == oracle.alg2_global(g)
    assert np.array_equal(pe, oracle.alg2_per_edge(g))


@pytest.mark.parametrize("mode", ["pull_always", "pull_never", gd.GD_VARIANT_ORIENTED])
def test_bipartite_hubs_closed_form(ctxs, mode):
    """Complete bipartite graphs K_{a,b} (Table 1 counts in closed form): the
    b-side nodes are hubs whose masks are summed at the a-side nodes, whose
    degrees reach the warp path and, for K_{2,300000}, the path for
    degrees of 2^18 and more."""
    from test_oracle_pins import closed_bipartite
    for a, b in ((2, 300_000), (3, 70_000), (70, 1500)):
        g = inputs.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])
        with ctxs[mode].graph(g) as h:
            assert h.count_global() == closed_bipartite(a, b), (a, b)


@pytest.mark.parametrize("mode", ["pull_always", gd.GD_VARIANT_ORIENTED])
def test_per_edge_above_degree_65536(ctxs, mode):
    """Per-edge counts with a node of degree > 65536: the library keeps its
    per-slot 4-cycle credits in 64-bit words then (32-bit ones below, where
    no slot's total can reach 2^32).  Three hubs joined to 70,000 leaves that
    also form a random graph of their own, against the O2 oracle per edge."""
    rng = np.random.default_rng(17)
    leaves = 70_000
    edges = [(h, 3 + j) for h in range(3) for j in range(leaves)]
    a = rng.integers(0, leaves, 140_000)
    b = rng.integers(0, leaves, 140_000)
    edges += [(3 + int(x), 3 + int(y)) for x, y in zip(a, b) if x != y]
    g = inputs.from_edges(3 + leaves, edges)
    assert int(np.diff(g.row_ptr).max()) > 65536
    with ctxs[mode].graph(g) as h:
        pe, glob = h.count_per_edge()
    assert glob == oracle.o2_global(g)
    assert np.array_equal(pe, oracle.o2_per_edge(g))


def test_repeated_calls_identical(ctxs):
    g = inputs.barabasi_albert(5000, 4, 9)
    with ctxs[gd.GD_VARIANT_ORIENTED].graph(g) as h:
        a = [h.count_global() for _ in range(3)]
        b = [h.count_per_edge()[0] for _ in range(2)]
    assert a[0] == a[1] == a[2]
    assert np.array_equal(b[0], b[1])


def test_device_pointers_and_device_output(ctxs):
    torch = pytest.importorskip("torch")
    g = inputs.chung_lu(30_000, 2.3, 150_000, 0.0, 11)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    ctx = ctxs[gd.GD_VARIANT_ORIENTED]
    out = torch.empty((g.m, 15), dtype=torch.int64, device="cuda")
    for borrow in (False, True):
        with ctx.graph(rp, ci, n=g.n, borrow=borrow, validate=True) as h:
            _, glob = h.count_per_edge(out=out)
            torch.cuda.synchronize()
            pe = out.cpu().numpy().view(np.uint64)
    assert glob == oracle.o2_global(g)
    assert np.array_equal(pe, oracle.o2_per_edge(g))


def test_invalid_csr_rejected(ctxs):
    ctx = ctxs[gd.GD_VARIANT_ORIENTED]
    g = inputs.erdos_renyi(50, 0.2, 4)
    cases = []
    bad = g.col_idx.copy(); bad[0] = bad[1]                 # duplicate / unsorted
    cases.append((g.row_ptr, bad))
    bad = g.col_idx.copy(); bad[0] = 0                      # self-loop on node 0
    cases.append((g.row_ptr, bad))
    bad = g.col_idx.copy(); bad[-1] = 50                    # id out of range
    cases.append((g.row_ptr, bad))
    # asymmetric: drop one direction of the first edge, keep nnz even by dropping another
    e = g.edges()
    el = [tuple(x) for x in e[1:]]
    h = inputs.from_edges(50, el)
    u, v = int(e[0][0]), int(e[0][1])
    ci = list(h.col_idx)
    rp = h.row_ptr.copy()
    # insert v into row u only, remove the last entry of the last non-empty row
    pos = int(rp[u]) + int(np.searchsorted(h.col_idx[rp[u]:rp[u + 1]], v))
    ci.insert(pos, v)
    rp[u + 1:] += 1
    last = max(i for i in range(50) if rp[i + 1] > rp[i])
    del ci[int(rp[last + 1]) - 1]
    rp[last + 1:] -= 1
    cases.append((rp, np.array(ci, dtype=np.int32)))
    # two entries below the diagonal without reverses (every entry above it
    # keeps its reverse; only the counts above and below differ)
    adj = [set(g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]].tolist()) for i in range(50)]
    extra = [(x, y) for x in range(49, 0, -1) for y in range(x) if y not in adj[x]][:2]
    assert len(extra) == 2
    for x, y in extra:
        adj[x].add(y)
    rows = [sorted(a) for a in adj]
    rp2 = np.zeros(51, dtype=np.int32)
    rp2[1:] = np.cumsum([len(r) for r in rows])
    cases.append((rp2, np.array([v for r in rows for v in r], dtype=np.int32)))
    for rp_, ci_ in cases:
        with pytest.raises(gd.GDError) as ei:
            ctx.graph(np.asarray(rp_, np.int32), np.asarray(ci_, np.int32), n=50, validate=True)
        assert ei.value.code == gd.GD_EINVAL
    # row_ptr that does not start at 0 is refused even without validation
    with pytest.raises(gd.GDError):
        ctx.graph(g.row_ptr + 1, g.col_idx, n=50)
    # row_ptr decreasing at one row, both ends intact: refused from host
    # arrays (host check) and from device arrays (device check)
    u = next(i for i in range(1, 49) if g.row_ptr[i + 1] > g.row_ptr[i])
    bad_rp = g.row_ptr.copy()
    bad_rp[u], bad_rp[u + 1] = bad_rp[u + 1], bad_rp[u]
    with pytest.raises(gd.GDError) as ei:
        ctx.graph(bad_rp, g.col_idx, n=50)
    assert ei.value.code == gd.GD_EINVAL and f"row {u}" in str(ei.value)
    torch = pytest.importorskip("torch")
    with pytest.raises(gd.GDError) as ei:
        ctx.graph(torch.from_numpy(bad_rp).cuda(), torch.from_numpy(g.col_idx).cuda(), n=50)
    assert ei.value.code == gd.GD_EINVAL
    with ctx.graph(g) as h:                      # the context stays usable
        assert h.count_global() == bruteforce.global_counts(g)


def test_budget_refusal():
    g = inputs.erdos_renyi(2000, 0.01, 3)
    with gd.Context(0, hbm_budget_bytes=4096) as c:
        with pytest.raises(gd.GDError) as ei:
            with c.graph(g) as h:
                h.count_global()
        assert ei.value.code == gd.GD_ENOMEM


def _golden(name):
    if not os.path.exists(GOLDEN):
        pytest.skip("golden workload counts not generated")
    with open(GOLDEN) as f:
        data = json.load(f)
    if name not in data:
        pytest.skip(f"no golden counts for {name}")
    return data[name]


def _csr_sha(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.col_idx, dtype="<i4").tobytes())
    return h.hexdigest()


@pytest.fixture(scope="module")
def chung_lu():
    return inputs.chung_lu_1m()


def test_chung_lu_workload_global_and_per_edge(ctxs, chung_lu):
    """Chung-Lu n=1M, ~10M edges: global counts and the full per-edge matrix
    (by digest) against the O2 oracle, plus sampled edges recomputed live by
    the O1 per-edge record."""
    rec = _golden("chung_lu_1m")
    g = chung_lu
    assert _csr_sha(g) == rec["csr_sha256"], "generator produced a different graph"
    ctx = ctxs[gd.GD_VARIANT_ORIENTED]
    with ctx.graph(g) as h:
        glob = h.count_global()
        pe, glob2 = h.count_per_edge()
    want = [int(x) for x in rec["global"]]
    assert glob == want and glob2 == want
    assert hashlib.sha256(np.ascontiguousarray(pe, dtype="<u8").tobytes()).hexdigest() == rec["per_edge_sha256"]
    # sampled edges, recomputed one by one from the definitions
    e = g.edges()
    rng = np.random.default_rng(123)
    deg = g.degrees()
    idx = rng.choice(len(e), 40, replace=False)
    small = np.flatnonzero((deg[e[:, 0]] < 200) & (deg[e[:, 1]] < 200))
    idx = np.concatenate([idx, rng.choice(small, 60, replace=False), hub_edges(g, e, pe, rng)])
    assert np.array_equal(pe[idx], oracle.edges_direct(g, e[idx]))


def hub_edges(g, e, pe, rng, each=20, hubs=8):
    """Edges where the hub tiers do their work: the largest d_u + d_v, the
    largest |Tri_e| (column g31), and edges at the highest-degree nodes."""
    deg = g.degrees()
    dsum = deg[e[:, 0]] + deg[e[:, 1]]
    by_deg = np.argsort(-dsum, kind="stable")[:each]
    by_tri = np.argsort(-pe[:, 0].astype(np.int64), kind="stable")[:each]
    top = np.argsort(-deg, kind="stable")[:hubs]
    at_hub = np.flatnonzero(np.isin(e[:, 0], top) | np.isin(e[:, 1], top))
    return np.unique(np.concatenate([by_deg, by_tri, rng.choice(at_hub, each, replace=False)]))


def test_rmat_workload_global_and_per_edge(ctxs):
    """R-MAT scale 22 (64M edges, hubs of degree 1.6e5): global counts
    against the O2 oracle (stored), the full per-edge matrix against them
    through the subset-count invariant, and sampled edges -- hub edges
    included -- against the O1 per-edge record."""
    rec = _golden("rmat_22")
    g = inputs.rmat_22()
    assert _csr_sha(g) == rec["csr_sha256"], "generator produced a different graph"
    with ctxs[gd.GD_VARIANT_ORIENTED].graph(g) as h:
        glob = h.count_global()
        pe, glob2 = h.count_per_edge()
    want = [int(x) for x in rec["global"]]
    assert glob == want and glob2 == want
    edges_of = [3, 2, 1, 0, 6, 5, 4, 4, 3, 3, 3, 2, 2, 1, 0]
    for c in range(15):
        col = pe[:, c].astype(np.uint64)
        # exact: two 32-bit halves, each summed below 2^58
        total = (int((col >> np.uint64(32)).sum(dtype=np.uint64)) << 32) + \
            int((col & np.uint64(0xFFFFFFFF)).sum(dtype=np.uint64))
        assert total == edges_of[c] * want[c], c
    e = g.edges()
    rng = np.random.default_rng(321)
    idx = np.concatenate([rng.choice(len(e), 60, replace=False), hub_edges(g, e, pe, rng)])
    assert np.array_equal(pe[idx], oracle.edges_direct(g, e[idx]))


def test_autotune_keeps_counts_and_caches(tmp_path):
    from paper_1506_04322_gb300 import autotune
    g = inputs.chung_lu(60_000, 2.1, 420_000, 0.0, 31)
    with gd.Context(0) as ctx, ctx.graph(g) as h:
        before = h.count_global()
        pe_before, _ = h.count_per_edge()
        cache = str(tmp_path / "tune.json")
        r = autotune.tuned_options(ctx, h, g, per_edge=False, cache_path=cache, max_trials=6)
        assert not r["cached"] and r["trials"] >= 2 and r["best_ms"] <= r["default_ms"]
        assert h.count_global() == before
        assert np.array_equal(h.count_per_edge()[0], pe_before)
        r2 = autotune.tuned_options(ctx, h, g, per_edge=False, cache_path=cache)
        assert r2["cached"] and r2["options"] == r["options"]
        assert h.count_global() == before
