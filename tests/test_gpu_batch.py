"""GPU parity of the batched path (gd_count_batch) against the CPU oracle:
per-graph global counts, bit-exact, in one call."""
import numpy as np
import pytest

from oracle import oracle
from paper_1506_04322_gb300 import gd, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gd.Context(0)
    yield c
    c.close()


def expected(graphs):
    return np.array([oracle.alg2_global(g) for g in graphs], dtype=object)


def check(ctx, graphs, **kw):
    b = inputs.pack(graphs)
    got = ctx.count_batch(b, **kw)
    got = np.asarray(got).astype(np.uint64) if not hasattr(got, "cpu") else got.cpu().numpy().view(np.uint64)
    want = expected(graphs)
    for i, g in enumerate(graphs):
        assert [int(x) for x in got[i]] == list(want[i]), (i, g.name)


def test_batch_recipe_graphs(ctx):
    """Graphs of the 20,000-graph recipe (ER and BA, n in [20, 500])."""
    check(ctx, [inputs.batch_graph(i) for i in range(400)])


def test_batch_edge_cases(ctx):
    gs = [inputs.from_edges(0, []), inputs.from_edges(1, []), inputs.from_edges(2, [(0, 1)]),
          inputs.from_edges(40, [(i, j) for i in range(40) for j in range(i + 1, 40)]),
          inputs.from_edges(33, [(0, i) for i in range(1, 33)]),
          inputs.erdos_renyi(512, 0.05, 3), inputs.erdos_renyi(513, 0.05, 4),   # 512-node variant edge
          inputs.erdos_renyi(1024, 0.02, 5),
          inputs.erdos_renyi(1100, 0.01, 6),          # above the shared-memory limit: single-graph path
          inputs.from_edges(7, [])]
    check(ctx, gs)


def test_batch_device_pointers(ctx):
    torch = pytest.importorskip("torch")
    gs = [inputs.batch_graph(i, seed=9) for i in range(200)]
    b = inputs.pack(gs)
    db = inputs.PackedBatch(b.num_graphs, torch.from_numpy(b.graph_node_ptr).cuda(),
                            torch.from_numpy(b.row_ptr).cuda(), torch.from_numpy(b.col_idx).cuda())
    got = ctx.count_batch(db, device_out=True)
    torch.cuda.synchronize()
    got = got.cpu().numpy().view(np.uint64)
    want = expected(gs)
    for i in range(len(gs)):
        assert [int(x) for x in got[i]] == list(want[i])


def test_batch_repeated_calls(ctx):
    gs = [inputs.batch_graph(i, seed=12) for i in range(300)]
    b = inputs.pack(gs)
    a1 = np.array(ctx.count_batch(b))
    a2 = np.array(ctx.count_batch(b))
    assert np.array_equal(a1, a2)


def test_batch_rejects_edge_across_graphs(ctx):
    # two graphs on nodes {0,1} and {2,3}; edge (1,2) crosses the boundary
    g = inputs.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    b = inputs.PackedBatch(2, np.array([0, 2, 4], np.int32), g.row_ptr, g.col_idx)
    with pytest.raises(gd.GDError) as ei:
        ctx.count_batch(b)
    assert ei.value.code == gd.GD_EINVAL


def test_batch_captured_graph_replays(ctx):
    """GD_CAPTURE: the device part runs as a captured CUDA graph, replayed
    while the call is unchanged and re-captured when the offsets change."""
    torch = pytest.importorskip("torch")
    gs = [inputs.batch_graph(i, seed=21) for i in range(150)]
    b = inputs.pack(gs)
    db = inputs.PackedBatch(b.num_graphs, torch.from_numpy(b.graph_node_ptr).cuda(),
                            torch.from_numpy(b.row_ptr).cuda(), torch.from_numpy(b.col_idx).cuda())
    out = torch.empty((b.num_graphs, 15), dtype=torch.int64, device="cuda")
    want = np.array(ctx.count_batch(b))
    for _ in range(3):
        out.fill_(-1)
        ctx.count_batch(db, out=out, capture=True)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
    # another batch in the same buffers' shape but different graphs: re-captured
    gs2 = [inputs.batch_graph(i, seed=22) for i in range(150)]
    b2 = inputs.pack(gs2)
    db2 = inputs.PackedBatch(b2.num_graphs, torch.from_numpy(b2.graph_node_ptr).cuda(),
                             torch.from_numpy(b2.row_ptr).cuda(), torch.from_numpy(b2.col_idx).cuda())
    out2 = torch.empty((b2.num_graphs, 15), dtype=torch.int64, device="cuda")
    ctx.count_batch(db2, out=out2, capture=True)
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy().view(np.uint64), np.array(ctx.count_batch(b2)))


def _device_graphs(torch, graphs):
    return [(torch.from_numpy(g.row_ptr).cuda(),
             torch.from_numpy(g.col_idx if g.nnz else np.zeros(0, np.int32)).cuda()) for g in graphs]


@pytest.mark.parametrize("capture", [False, True])
def test_batch_gather_from_separate_device_csrs(ctx, capture):
    """gd_count_batch_gather: graphs that sit in device memory one by one are
    packed on the device by one gather kernel and counted in the batched
    launch; with GD_CAPTURE the gather, validation and count replay as one
    captured CUDA graph, and a change of graphs re-captures."""
    torch = pytest.importorskip("torch")
    gs = [inputs.batch_graph(i, seed=31) for i in range(120)]
    gs += [inputs.from_edges(0, []), inputs.from_edges(3, [(0, 1)]),
           inputs.from_edges(30, [(i, j) for i in range(30) for j in range(i + 1, 30)])]
    if not capture:
        gs.append(inputs.erdos_renyi(1100, 0.01, 6))      # above the shared-memory limit
    dg = _device_graphs(torch, gs)
    want = expected(gs)
    for _ in range(3 if capture else 1):
        got = ctx.count_batch_gather(dg, capture=capture)
        torch.cuda.synchronize()
        got = got.cpu().numpy().view(np.uint64)
        for i in range(len(gs)):
            assert [int(x) for x in got[i]] == list(want[i]), (i, gs[i].name)
    gs2 = [inputs.batch_graph(i, seed=32) for i in range(123)]
    got2 = ctx.count_batch_gather(_device_graphs(torch, gs2), capture=capture)
    torch.cuda.synchronize()
    want2 = expected(gs2)
    got2 = got2.cpu().numpy().view(np.uint64)
    for i in range(len(gs2)):
        assert [int(x) for x in got2[i]] == list(want2[i])


def test_batch_gather_rejects_bad_row_ptr(ctx):
    torch = pytest.importorskip("torch")
    g = inputs.erdos_renyi(40, 0.2, 3)
    rp = g.row_ptr.copy()
    rp[0] = 1
    dg = [(torch.from_numpy(rp).cuda(), torch.from_numpy(g.col_idx).cuda())]
    with pytest.raises(gd.GDError) as ei:
        ctx.count_batch_gather(dg)
    assert ei.value.code == gd.GD_EINVAL
    # the context stays usable
    got = ctx.count_batch_gather(_device_graphs(torch, [g]))
    torch.cuda.synchronize()
    assert [int(x) for x in got.cpu().numpy().view(np.uint64)[0]] == list(expected([g])[0])


def test_batch_autotune_keeps_counts_and_caches(tmp_path):
    """gd_autotune_batch times the batched kernel's CTA sizes on a batch and
    keeps the fastest; the counts are the same under every choice, and the
    choice is cached by the batch's size signature."""
    from paper_1506_04322_gb300 import autotune
    gs = [inputs.batch_graph(i, seed=41) for i in range(300)] + [inputs.erdos_renyi(900, 0.01, 2)]
    b = inputs.pack(gs)
    want = expected(gs)
    with gd.Context(0) as c:
        cache = str(tmp_path / "tune.json")
        r = autotune.tuned_batch_options(c, b, cache_path=cache)
        assert not r["cached"] and r["trials"] >= 3 and r["best_ms"] <= r["default_ms"]
        assert c.options().batch_threads == r["options"]["batch_threads"]
        got = np.array(c.count_batch(b))
        for i in range(len(gs)):
            assert [int(x) for x in got[i]] == list(want[i])
        r2 = autotune.tuned_batch_options(c, b, cache_path=cache)
        assert r2["cached"] and r2["options"] == r["options"]
        for t in (128, 256, 512, 1024):
            o = c.options()
            o.batch_threads = t
            c.set_options(o)
            assert np.array_equal(np.array(c.count_batch(b)), got)
