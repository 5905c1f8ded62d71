"""GPU tests of the request loop (gd_submit / gd_poll): every result equals
the same graph counted alone, admission respects the device-memory budget,
requests overlap on the device, and a bad request fails alone."""
import time

import numpy as np
import pytest

from oracle import oracle
from paper_1506_04322_gb300 import gd, inputs

pytestmark = pytest.mark.gpu


def mixed_graphs(seed=0):
    gs = [inputs.batch_graph(i, seed=50 + seed) for i in range(40)]
    gs += [inputs.chung_lu(n, 2.0 + 0.2 * (k % 4), n * 6, 0.0, 900 + seed * 10 + k)
           for k, n in enumerate([3000, 12000, 40000, 5000, 90000, 2500, 20000, 60000])]
    gs += [inputs.from_edges(0, []), inputs.from_edges(5, [])]
    rng = np.random.default_rng(seed)
    return [gs[i] for i in rng.permutation(len(gs))]


def collect(ctx, ids, timeout_s=120):
    res = {}
    t_end = time.time() + timeout_s
    while len(res) < len(ids):
        assert time.time() < t_end, "requests did not finish"
        for rid in ids:
            if rid in res:
                continue
            rc, counts, st = ctx.poll(rid)
            if rc != gd.GD_EAGAIN:
                res[rid] = (rc, counts, st)
        time.sleep(0.002)
    return res


def test_results_same_alone_and_in_the_mix():
    gs = mixed_graphs()
    with gd.Context(0) as alone:
        want = []
        for g in gs:
            with alone.graph(g) as h:
                want.append(h.count_global())
    for g, w in zip(gs, want):
        if g.n <= 600:
            assert w == oracle.alg2_global(g)
    with gd.Context(0) as ctx:
        ctx.serve_start(slots=4)
        ids = [ctx.submit(g) for g in gs]
        res = collect(ctx, ids)
        for rid, w in zip(ids, want):
            rc, counts, st = res[rid]
            assert rc == gd.GD_OK
            assert counts == w
        stats = ctx.serve_stats()
        assert stats["batched_launches"] >= 1      # small requests rode together
        ctx.serve_stop()


def test_admission_respects_the_budget():
    gs = [inputs.chung_lu(n, 2.2, n * 8, 0.0, 1700 + n) for n in (20000, 30000, 25000, 40000, 35000, 15000)]
    with gd.Context(0) as probe:
        fps = [probe.footprint_estimate(g.n, g.nnz) for g in gs]
    budget = int(max(fps) * 1.6)       # at most one large request at a time, sometimes two
    with gd.Context(0) as ctx:
        ctx.serve_start(slots=4, hbm_budget_bytes=budget)
        ids = [ctx.submit(g) for g in gs]
        res = collect(ctx, ids)
        spans = []
        for rid, g in zip(ids, gs):
            rc, counts, st = res[rid]
            assert rc == gd.GD_OK
            with gd.Context(0) as alone, alone.graph(g) as h:
                assert counts == h.count_global()
            spans.append((st["start_ms"], st["end_ms"], st["footprint"]))
        for t, _, _ in spans:                       # footprint admitted at each start
            live = sum(fp for s, e, fp in spans if s <= t < e)
            assert live <= budget
        # a request larger than the whole budget is refused at submission
        big = inputs.chung_lu(200000, 2.2, 1_600_000, 0.0, 3)
        with pytest.raises(gd.GDError) as ei:
            ctx.submit(big)
        assert ei.value.code == gd.GD_ENOMEM
        ctx.serve_stop()


def test_requests_overlap_on_the_device():
    gs = [inputs.chung_lu(60000, 2.1, 480000, 0.0, 2300 + k) for k in range(8)]
    with gd.Context(0) as ctx:
        ctx.serve_start(slots=4)
        ids = [ctx.submit(g) for g in gs]
        res = collect(ctx, ids)
        spans = sorted((st["start_ms"], st["end_ms"]) for rc, _, st in res.values())
        assert all(rc == gd.GD_OK for rc, _, _ in res.values())
        overlap = any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
        assert overlap
        assert len({st["slot"] for _, _, st in res.values()}) > 1
        ctx.serve_stop()


def test_bad_request_fails_alone():
    good = [inputs.chung_lu(8000, 2.3, 40000, 0.0, 4100 + k) for k in range(3)]
    g = inputs.erdos_renyi(3000, 0.003, 7)
    bad = inputs.Graph(g.n, g.row_ptr.copy(), g.col_idx.copy())
    bad.col_idx[0] = bad.col_idx[1]                 # repeated neighbour: not a simple graph
    with gd.Context(0) as ctx:
        ctx.serve_start(slots=2)
        ids = [ctx.submit(x) for x in (good[0], bad, good[1], good[2])]
        res = collect(ctx, ids)
        assert res[ids[1]][0] == gd.GD_EINVAL
        for rid, x in zip([ids[0], ids[2], ids[3]], good):
            rc, counts, _ = res[rid]
            assert rc == gd.GD_OK
            with gd.Context(0) as alone, alone.graph(x) as h:
                assert counts == h.count_global()
        ctx.serve_stop()


def test_large_request_is_not_starved():
    """A large request queued among many small ones, under a budget that it
    fits only while no small request is admitted: once it has been passed
    over for GD_SERVE_MAX_BYPASS_MS, admissions stop until it fits, so it
    finishes long before the small requests queued after it."""
    small = [inputs.chung_lu(4000, 2.3, 16000, 0.0, 5100 + k) for k in range(400)]
    large = inputs.chung_lu(60000, 2.1, 480000, 0.0, 5099)
    with gd.Context(0) as probe:
        fp_s = max(probe.footprint_estimate(g.n, g.nnz) for g in small)
        fp_l = probe.footprint_estimate(large.n, large.nnz)
    with gd.Context(0) as ctx:
        ctx.serve_start(slots=4, hbm_budget_bytes=fp_l + fp_s // 2)
        ids = [ctx.submit(g) for g in small[:20]]
        lid = ctx.submit(large)
        later = [ctx.submit(g) for g in small[20:]]
        res = collect(ctx, ids + [lid] + later)
        rc, counts, st = res[lid]
        assert rc == gd.GD_OK
        with gd.Context(0) as alone, alone.graph(large) as h:
            assert counts == h.count_global()
        before = sum(1 for r in later if res[r][2]["start_ms"] < st["start_ms"])
        assert before < len(later) // 2, f"{before} later requests started before the large one"
        assert st["end_ms"] - st["submit_ms"] < 2000
        assert all(res[r][0] == gd.GD_OK for r in ids + later)
        ctx.serve_stop()
