"""Benchmark: exact 3+4-node graphlet counts (global + per-edge) on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gd|reference]

One step = the whole single-graph path of libgd on the Chung-Lu workload
(n = 1,000,000, ~10M undirected edges, Pareto exponent 2.1, expected degree
capped at 50,000, seed 2): CSR ingest/schedule, Step 1 (|Tri_e| per edge),
node/triangle sums, Step 2 (4-cliques and 4-cycles), Step 3/4 per edge
(15 columns written to HBM) and the exact u128 global completion.

* ``value``  -- edges/s with the CSR resident in HBM (CUDA events on the
  library's stream, L2 flushed by a 512 MB write between timed steps).
* ``e2e``    -- the same metric through the C ABI with host buffers: upload the
  CSR from pinned host memory, count, copy the per-edge matrix and the global
  counts back to pinned host memory, release the graph.
* ``roofline`` -- the dominant kernel's algorithmic bytes per launch over its
  average CUDA-event duration (timed live in the timed region), against the
  measured HBM copy bandwidth.
* ``cpu_baseline`` -- the CPU oracle (per-edge records from the definitions,
  single thread) on a random sample of the same graph's edges.

Multi-GPU (torchrun): replicas only -- every rank counts its own copy of the
workload (weak scaling); there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1506_04322_gb300 import inputs  # noqa: E402

METRIC = "edges/sec (exact 3+4-node graphlet counts)"
UNIT = "edges/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gd", choices=["gd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--smem-table", type=int, default=None, help="gd_options.smem_table_max")
    ap.add_argument("--bitmap-max", type=int, default=None, help="gd_options.bitmap_max_outdeg")
    ap.add_argument("--hub-log2", type=int, default=None, help="gd_options.hub_wedges_log2")
    ap.add_argument("--hub-pull", type=int, default=None, help="gd_options.hub_pull (0 auto, 1 never, 2 always)")
    ap.add_argument("--medium-cl", type=int, default=None, help="gd_options.medium_cluster_log2 (above 40: never)")
    ap.add_argument("--global-only", action="store_true", help="time gd_count_global instead")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-graphs measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-loop measurement")
    ap.add_argument("--no-rmat", action="store_true", help="skip the R-MAT scale-22 global-count record")
    ap.add_argument("--no-variants", action="store_true", help="skip the literal-variant comparison")
    ap.add_argument("--serving-requests", type=int, default=1000, help="requests of the serving trace")
    ap.add_argument("--cpu-o2", action="store_true",
                    help="also time the O2 oracle on the whole graph with every host core (minutes)")
    ap.add_argument("--workload", default="chung_lu_1m", choices=["chung_lu_1m", "chung_lu_400k", "rmat_22", "rmat_20"],
                    help="chung_lu_400k: a 4M-edge graph of the same family, for profiler captures; "
                         "rmat_22: the R-MAT scale-22 graph (use with --global-only); rmat_20: R-MAT scale 20, "
                         "edge factor 16, for profiler captures of the global-count kernels")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (the slowest replica sets the job's
    time); x itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all replicas processed over the
    slowest replica's time."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic bytes (per kernel launch) from the CSR
# ---------------------------------------------------------------------------

KERNEL_FAMILIES = {
    # bitmap passes over N+(a): triangles + 4-cliques, and the triangle sums
    "bitmap": ("k_clique_bitmap", "k_trisum_bitmap"),
    # 4-cycle tiers: wedge walks (push) and, for global counts, the hub
    # batches in pull form
    "cycles": ("k_cycles_tiny", "k_cycles_small", "k_cycles_medium", "k_cycles_hub_count",
               "k_cycles_hub_credit", "k_cycles_hub_clear", "k_pull_mark", "k_pull_thread",
               "k_pull_warp", "k_pull_heavy", "k_pull_clear"),
}

PULL_MAX = 64


def algorithmic_bytes(g, triangles: int, per_edge: bool, pull_batches: int = 0, hub_log2: int = 17,
                      hub_batch: int = 16) -> dict:
    """Bytes each kernel family must move for this graph, per step (4-byte
    ids, degrees and |Tri| counters, 8-byte credits and masks).  Nodes are
    ranked by (degree, id); a -> c orients every edge from the lower-ranked
    end.

    bitmap (one pass for global counts, a second for the per-edge triangle
      sums): per pass the out-lists N+(a) (12 B per out-edge: id, slot,
      degree) and the out-lists of their members (4 B per entry,
      X = sum over out-edges a->c of |N+(c)|); per triangle the (b,c) slot
      lookup (8 B) and its credits (|Tri| 4 B + 4-clique 8 B in the first
      pass; three |Tri| reads 12 B + two 8 B credits in the second).
    cycles, push form (4-cycles counted from their top-ranked node u): every
      adjacency entry of u read once (id + degree, 8 B each, 16 B per edge);
      for every lower neighbour v the whole list N(v) scanned (8 B per entry,
      W = sum over edges of the smaller degree); one counter update per live
      wedge (y ranked below u; L wedges, 4 B).  The per-edge credit pass
      repeats the scan, reads each live counter (4 B), credits (v,y) and
      credits each (u,v) once (a credit word each: 4 B when the largest
      degree is at most 65536, as the library keeps them then, else 8 B).
    cycles, pull form (hub batches in decreasing rank: for global counts the
      first pull_batches batches of 64 hubs; for per-edge credits the batches
      of `hub_batch` hubs with at least 2 nnz wedges, whose counts the pull
      writes into the tables): per batch every CSR slot read once with its
      neighbour's 8-byte mask (12 B per slot), and the hubs' lists marked and
      cleared (24 B per entry); their wedges leave the push terms of the count
      pass (the per-edge credit pass walks every wedge as before).
    """
    d = g.degrees().astype(np.int64)
    n = g.n
    rank = np.empty(n, dtype=np.int64)
    rank[np.lexsort((np.arange(n), d))] = np.arange(n)
    rows = np.repeat(np.arange(n, dtype=np.int64), d)
    cols = g.col_idx.astype(np.int64)
    m = len(cols) // 2
    up = rank[cols] > rank[rows]                          # entry v -> u with u above v
    dplus = np.bincount(rows[up], minlength=n)
    X = int(dplus[cols[up]].sum())
    # per top node u: W(u) = sum of d_v over lower neighbours v, L(u) = the
    # members of those lists ranked below u (position of u in N(v) by rank)
    key = np.sort(rows * n + rank[cols])
    pos = np.arange(len(cols), dtype=np.int64) - g.row_ptr.astype(np.int64)[key // n]
    ranked = np.empty(n, dtype=np.int64)
    ranked[rank] = np.arange(n)
    cu = ranked[key % n]                                  # neighbour at each rank-ordered slot
    upk = rank[cu] > rank[key // n]
    Wu = np.bincount(cu[upk], weights=d[(key // n)[upk]], minlength=n).astype(np.int64)
    Lu = np.bincount(cu[upk], weights=pos[upk], minlength=n).astype(np.int64)
    W, L = int(Wu.sum()), int(Lu.sum())
    pull_bytes, Wp, Lp = 0, 0, 0
    if pull_batches:
        thr = max(1 << hub_log2, n // 8)
        hubs = np.flatnonzero(Wu > thr)
        hubs = hubs[np.lexsort((-hubs, -d[hubs]))]
        if per_edge:
            batches = [hubs[i:i + hub_batch] for i in range(0, len(hubs), hub_batch)]
            pulled = [b for b in batches if int(Wu[b].sum()) >= 2 * len(cols)]
            hubs = np.concatenate(pulled) if pulled else hubs[:0]
            npull = len(pulled)
        else:
            hubs = hubs[:PULL_MAX * pull_batches]
            npull = pull_batches
        Wp, Lp = int(Wu[hubs].sum()), int(Lu[hubs].sum())
        pull_bytes = npull * 12 * len(cols) + 24 * int(d[hubs].sum())
    passes = 2 if per_edge else 1
    bitmap = passes * (12 * m + 4 * X) + triangles * (20 + (36 if per_edge else 0))
    cycles = 16 * m + 8 * (W - Wp) + 4 * (L - Lp) + pull_bytes
    if per_edge:
        cw = 4 if int(d.max(initial=0)) <= 65536 else 8     # credit words (32-bit below degree 2^16)
        cycles += 16 * m + 8 * W + (4 + cw) * L + cw * m
    return {"bitmap": bitmap, "cycles": cycles, "W": W, "L": L, "X": X, "m": m,
            "pulled_hub_wedges": Wp, "pull_batches": npull if pull_batches else 0}


def source_digest() -> str:
    """Digest of the sources of the bitmap and 4-cycle kernels (the families
    whose DRAM traffic is taken from a committed ncu summary)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1506_04322_gb300", "csrc")
    for f in ("gd_step2.cu", "gd_device.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, family: str):
    """DRAM bytes per step of a kernel family from the committed ncu summary
    of this workload, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    if t.get("source_digest") != source_digest():
        return None
    return t.get("families", {}).get(family)


def run_batch_measure(gd, torch, ctx, device, steps: int, loop_graphs: int = 600) -> dict:
    """Batched counting of the 20,000-graph recipe (one persistent launch per
    call) against a per-graph loop of the single-graph path on the same GPU."""
    gs = inputs.graph_batch(20_000)
    b = inputs.pack(gs)
    G = b.num_graphs
    db = inputs.PackedBatch(G, torch.from_numpy(b.graph_node_ptr).to(device),
                            torch.from_numpy(b.row_ptr).to(device), torch.from_numpy(b.col_idx).to(device))
    out = torch.empty((G, 15), dtype=torch.int64, device=device)
    for _ in range(3):
        ctx.count_batch(db, out=out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.count_batch(db, out=out)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    res = out.cpu().numpy().view(np.uint64)
    # the same call replayed as a captured CUDA graph (validate -> count)
    outc = torch.empty((G, 15), dtype=torch.int64, device=device)
    for _ in range(3):
        ctx.count_batch(db, out=outc, capture=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.count_batch(db, out=outc, capture=True)
    torch.cuda.synchronize()
    dt_cap = (time.perf_counter() - t0) / steps
    if not np.array_equal(outc.cpu().numpy().view(np.uint64), res):
        raise RuntimeError("captured batch counts differ")
    # graphs held one by one on the device: gather -> validate -> count as one
    # captured CUDA graph (gd_count_batch_gather)
    dg = [(torch.from_numpy(g.row_ptr).to(device),
           torch.from_numpy(g.col_idx if g.nnz else np.zeros(0, np.int32)).to(device)) for g in gs]
    outg = torch.empty((G, 15), dtype=torch.int64, device=device)
    rps = torch.tensor([r.data_ptr() for r, _ in dg], dtype=torch.int64, device=device)
    cis = torch.tensor([c.data_ptr() for _, c in dg], dtype=torch.int64, device=device)
    nn = np.array([g.n for g in gs], dtype=np.int32)
    ns = np.array([g.nnz for g in gs], dtype=np.int64)
    torch.cuda.synchronize()

    def gather_call():
        gd.gd_count_batch_gather(ctx.handle, G, rps.data_ptr(), cis.data_ptr(), nn.ctypes.data, ns.ctypes.data,
                                 gd.GD_CAPTURE, outg.data_ptr())

    for _ in range(3):
        gather_call()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        gather_call()
    torch.cuda.synchronize()
    dt_gather = (time.perf_counter() - t0) / steps
    if not np.array_equal(outg.cpu().numpy().view(np.uint64), res):
        raise RuntimeError("gathered batch counts differ")
    del dg
    # end to end from pinned host memory
    hb = inputs.PackedBatch(G, torch.from_numpy(b.graph_node_ptr).pin_memory().numpy(),
                            torch.from_numpy(b.row_ptr).pin_memory().numpy(),
                            torch.from_numpy(b.col_idx).pin_memory().numpy())
    hout = np.zeros((G, 15), dtype=np.uint64)
    ctx.count_batch(hb, out=hout)
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.count_batch(hb, out=hout)
    dt_e2e = (time.perf_counter() - t0) / steps
    if not np.array_equal(hout, res):
        raise RuntimeError("batched counts differ between device and host inputs")
    # per-graph loop: device-resident CSR per graph, one gd_count_global each
    sub = gs[:loop_graphs]
    dev = [(torch.from_numpy(g.row_ptr).to(device), torch.from_numpy(g.col_idx if g.nnz else np.zeros(1, np.int32)).to(device), g)
           for g in sub]
    torch.cuda.synchronize()
    loop_res = []
    t0 = time.perf_counter()
    for rp, ci, g in dev:
        h = gd.gd_create_csr(ctx.handle, g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), gd.GD_DEVICE_PTRS | gd.GD_BORROW, 0)
        loop_res.append(gd.gd_count_global(ctx.handle, h))
        gd.gd_destroy_graph(h)
    torch.cuda.synchronize()
    dt_loop = (time.perf_counter() - t0) / len(sub)
    for i, r in enumerate(loop_res):
        if [int(x) for x in res[i]] != r:
            raise RuntimeError(f"batched and per-graph counts differ on graph {i}")
    # graphlet frequency features of every graph of the batch (17 doubles each)
    feats = torch.empty((G, 17), dtype=torch.float64, device=device)
    gd.gd_gfd_batch(ctx.handle, G, db.graph_node_ptr.data_ptr(), db.row_ptr.data_ptr(), out.data_ptr(), feats.data_ptr())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        gd.gd_gfd_batch(ctx.handle, G, db.graph_node_ptr.data_ptr(), db.row_ptr.data_ptr(), out.data_ptr(),
                        feats.data_ptr())
    torch.cuda.synchronize()
    dt_gfd = (time.perf_counter() - t0) / steps
    return {"workload": "graph_batch_20000 (n~U[20,500], half ER mean degree U[2,12], half BA m in {1,2,3})",
            "graphs": G, "nodes": int(b.graph_node_ptr[-1]), "edges": int(b.row_ptr[-1]) // 2,
            "graphs_per_s": G / dt, "ms_per_batch": 1000 * dt, "e2e_graphs_per_s": G / dt_e2e,
            "captured_graphs_per_s": G / dt_cap, "captured_ms_per_batch": 1000 * dt_cap,
            "gather_captured_graphs_per_s": G / dt_gather, "gather_captured_ms_per_batch": 1000 * dt_gather,
            "per_graph_loop_graphs_per_s": 1.0 / dt_loop, "per_graph_loop_sample": len(sub),
            "speedup_vs_loop": (G / dt) * dt_loop,
            "features_ms_per_batch": 1000 * dt_gfd, "features_graphs_per_s": G / dt_gfd}


def run_next_measure(gd, torch, ctx, h, g, out) -> dict:
    """Edge insert/delete updates and ranking on the single-graph workload:
    toggles per second (random edges, random non-edges, pairs of hubs)
    against one full global recount, and top-k / node-sum times over the
    per-edge matrix already in HBM."""
    rng = np.random.default_rng(8)
    e = g.edges()
    deg = g.degrees()
    hubs = np.argsort(-deg)[:8]
    pairs = [tuple(int(x) for x in e[i]) for i in rng.choice(len(e), 100, replace=False)]
    pairs += [(int(a), int(b)) for a, b in rng.integers(0, g.n, size=(100, 2)) if a != b]
    hub_pairs = [(int(hubs[i]), int(hubs[j])) for i in range(8) for j in range(i + 1, 8)]
    h.toggle_delta(*pairs[0])
    t0 = time.perf_counter()
    for u, v in pairs:
        h.toggle_delta(u, v)
    dt_pair = (time.perf_counter() - t0) / len(pairs)
    t0 = time.perf_counter()
    for u, v in hub_pairs:
        h.toggle_delta(u, v)
    dt_hub = (time.perf_counter() - t0) / len(hub_pairs)
    h.count_global()
    t0 = time.perf_counter()
    h.count_global()
    dt_full = time.perf_counter() - t0
    ctx.topk(out, 1000, column=4)
    t0 = time.perf_counter()
    for _ in range(5):
        ctx.topk(out, 1000, column=4)
    dt_topk = (time.perf_counter() - t0) / 5
    node = torch.empty(g.n, dtype=torch.int64, device=out.device)
    h.node_sums(out, 0, out=node)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        h.node_sums(out, 0, out=node)
    torch.cuda.synchronize()
    dt_node = (time.perf_counter() - t0) / 5
    return {"toggle_ms_random_pair": 1000 * dt_pair, "toggle_ms_hub_pair": 1000 * dt_hub,
            "full_global_recount_ms": 1000 * dt_full, "toggles_per_s": 1.0 / dt_pair,
            "topk1000_ms_4clique_column": 1000 * dt_topk, "node_sums_ms": 1000 * dt_node,
            "pairs": f"{len(pairs)} random (100 edges, the rest non-edges), {len(hub_pairs)} pairs of the 8 largest hubs"}


def run_serving_measure(gd, count: int = 1000, loads=(0.3, 0.5, 0.7, 0.9), slots: int = 4, seed: int = 5) -> dict:
    """Request loop on the serving-trace recipe: Chung-Lu requests with m
    log-uniform on [1e3, 5e6], exponent U[2.0, 2.8].  Capacity from a closed
    loop (all requests submitted at once), then Poisson arrivals at each
    load x capacity; latency = completion - arrival.  Baseline at every load:
    the same arrivals served by a plain FIFO queue, one request at a time
    (gd_count_global per request).  Every served result is checked against
    the same graph counted alone."""
    import concurrent.futures as cf
    reqs = inputs.request_trace(count, rate_per_s=1.0, seed=seed)
    with cf.ThreadPoolExecutor(max_workers=max(4, (os.cpu_count() or 8))) as ex:
        graphs = list(ex.map(lambda r: r.graph(), reqs))
    edges = sum(g.m for g in graphs)

    def wait_all(ctx, ids):
        out = {}
        while len(out) < len(ids):
            for rid in ids:
                if rid not in out:
                    rc, counts, st = ctx.poll(rid)
                    if rc != gd.GD_EAGAIN:
                        if rc != gd.GD_OK:
                            raise RuntimeError(f"request failed: {rc}")
                        out[rid] = (counts, st)
            time.sleep(0.0005)
        return out

    # counts of every request alone, and the FIFO queue's service times
    alone = []
    with gd.Context(0) as ctx:
        for g in graphs[:4]:
            with ctx.graph(g) as h:
                h.count_global()
        service = []
        for g in graphs:
            t0 = time.perf_counter()
            with ctx.graph(g) as h:
                alone.append(h.count_global())
            service.append(time.perf_counter() - t0)
    fifo_capacity = count / sum(service)

    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0, size=count)       # unit-rate Poisson gaps, scaled per load
    points = []
    with gd.Context(0) as ctx:
        ctx.serve_start(slots=slots)
        wait_all(ctx, [ctx.submit(g) for g in graphs[:8]])          # warm-up
        t0 = time.perf_counter()
        ids = [ctx.submit(g) for g in graphs]
        closed = wait_all(ctx, ids)
        t_closed = time.perf_counter() - t0
        capacity = count / t_closed
        if [closed[r][0] for r in ids] != alone:
            raise RuntimeError("a served result differs from the same graph counted alone")
        for load in loads:
            rate = load * capacity
            arrivals = np.cumsum(gaps / rate)
            ids = []
            t0 = time.perf_counter()
            for a, g in zip(arrivals, graphs):
                dt = a - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                ids.append(ctx.submit(g))
            res = wait_all(ctx, ids)
            span = time.perf_counter() - t0
            if [res[r][0] for r in ids] != alone:
                raise RuntimeError("a served result differs from the same graph counted alone")
            lat = np.array([res[r][1]["end_ms"] - res[r][1]["submit_ms"] for r in ids])
            points.append({"load": load, "offered_req_per_s": rate, "throughput_req_per_s": count / span,
                           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))})
        stats = ctx.serve_stats()
        ctx.serve_stop()
    # FIFO queue on the same arrivals, run for real: one request at a time
    with gd.Context(0) as ctx:
        for g in graphs[:4]:
            with ctx.graph(g) as h:
                h.count_global()
        for pt in points:
            arrivals = np.cumsum(gaps / pt["offered_req_per_s"])
            fl = []
            t0 = time.perf_counter()
            for a, g, w in zip(arrivals, graphs, alone):
                now = time.perf_counter() - t0
                if now < a:
                    time.sleep(a - now)
                with ctx.graph(g) as h:
                    if h.count_global() != w:
                        raise RuntimeError("FIFO counts differ")
                fl.append(1000 * (time.perf_counter() - t0 - a))
            span = time.perf_counter() - t0
            pt.update({"fifo_throughput_req_per_s": count / span, "fifo_p50_ms": float(np.percentile(fl, 50)),
                       "fifo_p99_ms": float(np.percentile(fl, 99))})
    return {"workload": f"request trace: {count} Chung-Lu requests, m log-uniform [1e3,5e6], "
                        f"exponent U[2.0,2.8], n=max(32,m/8), seed {seed}",
            "requests": count, "edges": int(edges), "slots": slots,
            "capacity_req_per_s": capacity, "capacity_edges_per_s": edges / t_closed,
            "fifo_capacity_req_per_s": fifo_capacity,
            "sweep": points, "batched_launches": stats["batched_launches"],
            "single_launches": stats["single_launches"],
            "fifo_queue": "the same arrivals served one request at a time on one stream "
                          "(gd_create_csr + gd_count_global from host memory)",
            "results_identical_alone_and_in_mix": True}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle baseline
# ---------------------------------------------------------------------------

def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _o1_sample(g, e, order, seconds: float, threads: int) -> tuple[int, float]:
    """Per-edge O1 records of edges order[0], order[1], ... on `threads`
    host threads (the oracle's C calls release the interpreter lock) until
    `seconds` have passed; returns (edges done, wall seconds)."""
    import concurrent.futures as cf
    from oracle import oracle
    chunk = 16
    lock = threading.Lock()
    state = {"next": 0, "done": 0}
    t0 = time.perf_counter()

    def worker():
        while time.perf_counter() - t0 < seconds:
            with lock:
                i = state["next"]
                if i >= len(order):
                    return
                state["next"] = i + chunk
            idx = order[i:i + chunk]
            oracle.edges_direct(g, e[idx])
            with lock:
                state["done"] += len(idx)

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for f in [ex.submit(worker) for _ in range(threads)]:
            f.result()
    return state["done"], time.perf_counter() - t0


def cpu_baseline(g, seconds: float, seed: int = 0, one_thread_seconds: float = 3.0) -> dict:
    """The CPU oracle on the host's cores: per-edge counts from the
    definitions (O1 records, the paper's per-edge work of Algorithm 2) of
    uniformly random edges of the same graph, one edge per task on every
    core, as the paper's OpenMP loop over edges; and the same on one thread."""
    e = g.edges()
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(e))
    cores = os.cpu_count() or 1
    done, dt = _o1_sample(g, e, order, seconds, cores)
    rec = {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "cpu_model": cpu_model(), "nproc": cores, "_edges": done, "_seconds": dt,
           "sample": f"{done} uniformly random edges of the {g.m}-edge graph, per-edge counts from the "
                     f"definitions (O1 records), {cores} threads, {dt:.1f} s"}
    if one_thread_seconds > 0:
        done1, dt1 = _o1_sample(g, e, order[done:], one_thread_seconds, 1)
        rec["one_thread"] = {"value": done1 / dt1, "unit": UNIT, "edges": done1, "seconds": dt1}
    return rec


def cpu_o2(g) -> dict:
    """The independent oracle O2 (degree-ordered wedges, OpenMP) over the
    whole graph, global counts, every host core."""
    from oracle import oracle
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.o2_global(g, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": g.m / dt, "unit": UNIT, "seconds": dt, "threads": threads,
            "sample": f"whole graph ({g.m} edges), global counts"}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    g = inputs.chung_lu_1m()
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup):
        cpu_baseline(g, min(per_step, 2.0), seed=100 + i, one_thread_seconds=0)
    vals = [cpu_baseline(g, per_step, seed=i, one_thread_seconds=0) for i in range(args.steps)]
    total_edges = sum(v["_edges"] for v in vals)
    total_t = sum(v["_seconds"] for v in vals)
    value = total_edges / total_t
    cores = vals[0]["cores"] if vals else (os.cpu_count() or 1)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": g.name, "n": g.n, "m": g.m, "mode": "per-edge (15 columns) + global"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{int(total_edges)} uniformly random edges over {args.steps} steps, "
                                   f"O1 per-edge records on {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_workload(gd, torch, ctx, g, device, global_only: bool, steps: int, warmup: int, ws: int, rank: int,
                     hub_log2: int = 17) -> dict:
    """Time one workload: `steps` counts with the CSR resident in HBM (CUDA
    events on the library's stream, L2 flushed between steps, clocks
    sampled), then end to end through the C ABI from pinned host memory.
    Returns the record plus the live handles for follow-up measurements."""
    m = g.m
    stream = torch.cuda.Stream(device=device)
    rp = torch.from_numpy(g.row_ptr).to(device)
    ci = torch.from_numpy(g.col_idx).to(device)
    out = None if global_only else torch.empty((m, 15), dtype=torch.int64, device=device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)
    torch.cuda.synchronize()
    h = ctx.graph(rp, ci, n=g.n, borrow=True, stream=stream.cuda_stream)

    def step():
        if global_only:
            return h.count_global()
        return h.count_per_edge(out=out)[1]

    for _ in range(max(3, warmup)):
        with torch.cuda.stream(stream):
            flush.zero_()
        glob = step()
    torch.cuda.synchronize()

    clocks = ClockSampler(device)
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.kernel_launches()
    ctx.profile_begin()
    total_ms = 0.0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()                       # L2 flush, outside the timed events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        glob2 = step()
        with torch.cuda.stream(stream):
            e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        if glob2 != glob:
            raise RuntimeError("global counts changed between steps")
    prof = ctx.profile_end()
    launches = ctx.kernel_launches() - launches0
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if rank == 0 else None

    ms = max_over_ranks(total_ms / steps, device)
    value = job_rate(m, ws, ms / 1000.0)

    # end to end through the C ABI with pinned host buffers
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    ci_h = torch.from_numpy(g.col_idx).pin_memory()
    out_h = None if global_only else torch.empty((m, 15), dtype=torch.int64).pin_memory()
    h2d = 4 * (g.n + 1) + 4 * g.nnz
    d2h = (0 if global_only else 8 * 15 * m) + 16 * 15

    def e2e_step():
        gh = gd.gd_create_csr(ctx.handle, g.n, g.nnz, rp_h.data_ptr(), ci_h.data_ptr(), 0, stream.cuda_stream)
        try:
            if global_only:
                r = gd.gd_count_global(ctx.handle, gh)
            else:
                r = gd.gd_count_per_edge(ctx.handle, gh, out_h.data_ptr(), 0, True)
        finally:
            gd.gd_destroy_graph(gh)
        return r

    e2e_step()
    e2e_steps = max(2, min(steps, 5))
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r = e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if r != glob:
        raise RuntimeError("end-to-end counts differ from the device-resident counts")
    e2e_s = max_over_ranks(e2e_s, device)
    del rp_h, ci_h, out_h, flush

    kern = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1], "ms_total": v[0]} for k, v in prof.items()}
    rec = {"value": value, "ms_per_step": ms, "steps": steps, "warmup": max(3, warmup),
           "e2e": {"value": job_rate(m, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "gpu_launches": launches, "launches_before_timed": launches0, "clocks": clk,
           "kernels": {k: round(v["ms_total"] / steps, 3)
                       for k, v in sorted(kern.items(), key=lambda kv: -kv[1]["ms_total"])},
           "kernel_launches_per_step": {k: v["launches"] // steps for k, v in kern.items()},
           "global_counts": [str(x) for x in glob]}
    if rank == 0:
        peak, peak_kind = load_peaks()
        fam_ms = {f: sum(kern[k]["ms_total"] for k in names if k in kern) / steps
                  for f, names in KERNEL_FAMILIES.items()}
        dom = max(fam_ms, key=fam_ms.get)
        pull_batches = kern.get("k_pull_thread", {"launches": 0})["launches"] // steps
        hub_batch = max(1, min(16, (64 << 20) // (4 * max(g.n, 1))))
        ab = algorithmic_bytes(g, int(glob[0]), not global_only, pull_batches, hub_log2, hub_batch)
        if ab["pull_batches"] != pull_batches:
            raise RuntimeError("the byte model's pulled batches differ from the launched ones")
        achieved = ab[dom] / (fam_ms[dom] / 1000.0) / 1e9
        rec["roofline"] = {
            "kernel": dom, "kernels": [k for k in KERNEL_FAMILIES[dom] if k in kern], "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": measured_traffic(g.name, dom), "peak_kind": peak_kind,
            "algorithmic_bytes_per_step": ab[dom], "ms_per_step": fam_ms[dom],
            "per": "step (all launches of the family)",
            "units": {k: ab[k] for k in ("m", "W", "L", "X", "pulled_hub_wedges", "pull_batches")},
            "launches_per_step": sum(kern[k]["launches"] for k in KERNEL_FAMILIES[dom] if k in kern) // steps,
            "other_families": {f: {"ms_per_step": fam_ms[f], "algorithmic_bytes_per_step": ab[f],
                                   "achieved_gbs": ab[f] / (fam_ms[f] / 1000.0) / 1e9 if fam_ms[f] else None}
                               for f in fam_ms if f != dom}}
    return rec, h, out


def golden_counts(name: str):
    """Global counts of a workload stored by the oracle (tests/golden), if any."""
    p = os.path.join(ROOT, "tests", "golden", "workloads.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(name)
    return None if rec is None else [str(x) for x in rec["global"]]


def run_variants_measure(gd, torch, device, reps: int = 3) -> dict:
    """Degree-ordered pipeline (default) against the literal Algorithm 2
    kernels on the same graphs: global counts, device time per count."""
    out = {}
    for name, g in (("erdos_renyi_n2000_p0.005", inputs.erdos_renyi_small()),
                    ("chung_lu_n100k_gamma2.1_cap5k", inputs.chung_lu(100_000, 2.1, 1_100_000, 5_000.0, 9))):
        row = {"m": g.m}
        counts = {}
        for label, v in (("oriented", gd.GD_VARIANT_ORIENTED), ("literal", gd.GD_VARIANT_LITERAL)):
            with gd.Context(device, variant=v) as ctx, ctx.graph(g) as h:
                counts[label] = h.count_global()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(reps):
                    h.count_global()
                torch.cuda.synchronize()
                row[f"{label}_ms"] = 1000 * (time.perf_counter() - t0) / reps
        if counts["oriented"] != counts["literal"]:
            raise RuntimeError(f"variants disagree on {name}")
        row["literal_over_oriented"] = row["literal_ms"] / row["oriented_ms"]
        row["counts_equal"] = True
        out[name] = row
    return out


def run_gd(args):
    import torch
    from paper_1506_04322_gb300 import gd

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = local if ws > 1 else 0
    torch.cuda.set_device(device)
    if args.workload == "chung_lu_400k":
        g = inputs.chung_lu(400_000, 2.1, 4_400_000, 20_000.0, 9)
        g.name = "chung_lu_n400k_gamma2.1_cap20k"
    elif args.workload == "rmat_22":
        g = inputs.rmat_22()           # the global counts (per-edge output would be 7.7 GB)
    elif args.workload == "rmat_20":
        g = inputs.rmat(20, 16 << 20, 0.57, 0.19, 0.19, 3)
        g.name = "rmat_scale20_ef16"
    else:
        g = inputs.chung_lu_1m()

    ctx = gd.Context(device, smem_table_max=args.smem_table, bitmap_max_outdeg=args.bitmap_max,
                     hub_wedges_log2=args.hub_log2, hub_pull=args.hub_pull,
                     medium_cluster_log2=args.medium_cl)
    rec, h, out = measure_workload(gd, torch, ctx, g, device, args.global_only, args.steps, args.warmup,
                                   ws, rank, args.hub_log2 or 17)

    # the R-MAT scale-22 workload (global counts) in the same run
    rmat = None
    if args.workload == "chung_lu_1m" and not args.no_rmat:
        nxt0 = None
        if not args.global_only and not args.no_batch and rank == 0:
            nxt0 = run_next_measure(gd, torch, ctx, h, g, out)
        h.close()
        del out
        torch.cuda.empty_cache()
        gr = inputs.rmat_22()
        rmat, hr, _ = measure_workload(gd, torch, ctx, gr, device, True, max(2, min(args.steps, 5)),
                                       args.warmup, ws, rank, args.hub_log2 or 17)
        hr.close()
        want = golden_counts("rmat_22")
        rmat = {"workload": gr.name, "n": gr.n, "m": gr.m, "mode": "global", "metric": METRIC, "unit": UNIT,
                **rmat, "counts_equal_stored_oracle": None if want is None else want == rmat["global_counts"]}
        h = None
    else:
        nxt0 = None

    if rank != 0:
        if h is not None:
            h.close()
        ctx.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    nxt = nxt0
    if nxt is None and h is not None and not args.global_only and not args.no_batch:
        nxt = run_next_measure(gd, torch, ctx, h, g, out)
    batch = None
    if not args.no_batch:
        batch = run_batch_measure(gd, torch, ctx, device, max(2, min(args.steps, 5)))
    serving = None
    if not args.no_serving:
        serving = run_serving_measure(gd, count=args.serving_requests)
    variants = None
    if not args.no_variants:
        variants = run_variants_measure(gd, torch, device)

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(g, args.cpu_seconds)
        cpu = {k: v for k, v in cpu.items() if not k.startswith("_")}
        if args.cpu_o2:
            cpu["o2_all_cores"] = cpu_o2(g)

    line = {
        "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": g.name, "n": g.n, "m": g.m,
                   "mode": "global" if args.global_only else "per-edge (15 columns) + global",
                   "variant": "oriented", "seed": {"chung_lu_1m": 2, "chung_lu_400k": 9, "rmat_22": 3, "rmat_20": 3}[args.workload],
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{ws}"},
        "e2e": rec["e2e"],
        "gpu_launches": rec["gpu_launches"],
        "launches_before_timed": rec["launches_before_timed"],
        "roofline": rec.get("roofline"),
        "cpu_baseline": cpu,
        "clocks": rec["clocks"],
        "rmat_22": rmat,
        "batch": batch,
        "serving": serving,
        "variants": variants,
        "updates_and_ranking": nxt,
        "kernels": rec["kernels"],
        "kernel_launches_per_step": rec["kernel_launches_per_step"],
        "source_digest": source_digest(),
        "global_counts": rec["global_counts"],
    }
    print(json.dumps(line), flush=True)
    if h is not None:
        h.close()
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gd(args)


if __name__ == "__main__":
    main()
