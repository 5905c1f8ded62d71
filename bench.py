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
    ap.add_argument("--global-only", action="store_true", help="time gd_count_global instead")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-graphs measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-loop measurement")
    ap.add_argument("--workload", default="chung_lu_1m", choices=["chung_lu_1m", "chung_lu_400k", "rmat_22"],
                    help="chung_lu_400k: a 4M-edge graph of the same family, for profiler captures; "
                         "rmat_22: the R-MAT scale-22 graph (use with --global-only)")
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
    # 4-cycle tiers (wedge walks)
    "cycles": ("k_cycles_tiny", "k_cycles_small", "k_cycles_medium", "k_cycles_hub_count",
               "k_cycles_hub_credit", "k_cycles_hub_clear"),
}


def algorithmic_bytes(g, triangles: int, per_edge: bool) -> dict:
    """Bytes each kernel family must move for this graph, per step (4-byte
    ids, degrees and |Tri| counters, 8-byte credits).  Nodes are ranked by
    (degree, id); a -> c orients every edge from the lower-ranked end.

    bitmap (one pass for global counts, a second for the per-edge triangle
      sums): per pass the out-lists N+(a) (12 B per out-edge: id, slot,
      degree) and the out-lists of their members (4 B per entry,
      X = sum over out-edges a->c of |N+(c)|); per triangle the (b,c) slot
      lookup (8 B) and its credits (|Tri| 4 B + 4-clique 8 B in the first
      pass; three |Tri| reads 12 B + two 8 B credits in the second).
    cycles (4-cycles counted from their top-ranked node u): every adjacency
      entry of u read once (id + degree, 8 B each, 16 B per edge); for every
      lower neighbour v the whole list N(v) scanned (8 B per entry,
      W = sum over edges of the smaller degree); one counter update per live
      wedge (y ranked below u; L wedges, 4 B).  The per-edge credit pass
      repeats the scan, reads each live counter (4 B), credits (v,y) (8 B)
      and credits each (u,v) once (8 B).
    """
    d = g.degrees().astype(np.int64)
    n = g.n
    rank = np.empty(n, dtype=np.int64)
    rank[np.lexsort((np.arange(n), d))] = np.arange(n)
    rows = np.repeat(np.arange(n, dtype=np.int64), d)
    cols = g.col_idx.astype(np.int64)
    m = len(cols) // 2
    up = rank[cols] > rank[rows]                          # out-edge rows -> cols
    dplus = np.bincount(rows[up], minlength=n)
    X = int(dplus[cols[up]].sum())
    W = int(d[rows[up]].sum())                            # lower end's degree per edge
    # live wedges: for v and a higher neighbour u, the members of N(v) ranked below u
    order = np.lexsort((rank[cols], rows))
    pos = np.empty(len(cols), dtype=np.int64)
    pos[order] = np.arange(len(cols)) - g.row_ptr[rows[order]]
    L = int(pos[up].sum())
    passes = 2 if per_edge else 1
    bitmap = passes * (12 * m + 4 * X) + triangles * (20 + (36 if per_edge else 0))
    cycles = 16 * m + 8 * W + 4 * L
    if per_edge:
        cycles += 16 * m + 8 * W + 12 * L + 8 * m
    return {"bitmap": bitmap, "cycles": cycles, "W": W, "L": L, "X": X, "m": m}


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


def run_serving_measure(gd, count: int = 200, load: float = 0.7, slots: int = 4, seed: int = 5) -> dict:
    """Request loop on the serving-trace recipe: Chung-Lu requests with m
    log-uniform on [1e3, 5e6], exponent U[2.0, 2.8].  Capacity from a closed
    loop, then Poisson arrivals at `load` x capacity; latency = completion -
    arrival.  Baseline: the same arrivals served by a plain FIFO queue, one
    request at a time (gd_count_global per request)."""
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

    with gd.Context(0) as ctx:
        ctx.serve_start(slots=slots)
        wait_all(ctx, [ctx.submit(g) for g in graphs[:8]])          # warm-up
        t0 = time.perf_counter()
        ids = [ctx.submit(g) for g in graphs]
        closed = wait_all(ctx, ids)
        t_closed = time.perf_counter() - t0
        capacity = count / t_closed
        rate = load * capacity
        rng = np.random.default_rng(seed)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
        # open loop: submit at the arrival times
        ids = []
        t0 = time.perf_counter()
        for a, g in zip(arrivals, graphs):
            dt = a - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(ctx.submit(g))
        res = wait_all(ctx, ids)
        span = time.perf_counter() - t0
        lat = np.array([st["end_ms"] - st["submit_ms"] for _, st in res.values()])
        stats = ctx.serve_stats()
        results = [res[r][0] for r in ids]
        ctx.serve_stop()
    # baseline: FIFO queue, one request at a time, same arrivals
    with gd.Context(0) as ctx:
        for g in graphs[:4]:
            with ctx.graph(g) as h:
                h.count_global()
        t0 = time.perf_counter()
        base_lat = []
        for a, g, r in zip(arrivals, graphs, results):
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            with ctx.graph(g) as h:
                c = h.count_global()
            if c != r:
                raise RuntimeError("a served result differs from the same graph counted alone")
            base_lat.append(1000 * (time.perf_counter() - t0 - a))
        base_span = time.perf_counter() - t0
    base_lat = np.array(base_lat)
    return {"workload": f"request trace: {count} Chung-Lu requests, m log-uniform [1e3,5e6], "
                        f"exponent U[2.0,2.8], n=max(32,m/8), seed {seed}",
            "requests": count, "edges": int(edges), "slots": slots,
            "capacity_req_per_s": capacity, "capacity_edges_per_s": edges / t_closed,
            "offered_req_per_s": rate, "load": load,
            "throughput_req_per_s": count / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "batched_launches": stats["batched_launches"],
            "single_launches": stats["single_launches"],
            "fifo_queue": {"throughput_req_per_s": count / base_span,
                           "p50_ms": float(np.percentile(base_lat, 50)),
                           "p99_ms": float(np.percentile(base_lat, 99))},
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

def cpu_baseline(g, seconds: float, seed: int = 0) -> dict:
    from oracle import oracle
    e = g.edges()
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(e))
    done, t0 = 0, time.perf_counter()
    chunk = 16
    while time.perf_counter() - t0 < seconds and done < len(e):
        idx = order[done:done + chunk]
        oracle.edges_direct(g, e[idx])
        done += len(idx)
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "_edges": done, "_seconds": dt,
            "sample": f"{done} uniformly random edges of the {g.m}-edge graph, per-edge counts from the "
                      f"definitions (O1 record), one thread, {dt:.1f} s"}


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
        cpu_baseline(g, min(per_step, 2.0), seed=100 + i)
    vals = [cpu_baseline(g, per_step, seed=i) for i in range(args.steps)]
    total_edges = sum(v["_edges"] for v in vals)
    total_t = sum(v["_seconds"] for v in vals)
    value = total_edges / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": g.name, "n": g.n, "m": g.m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{int(total_edges)} random edges per run, O1 per-edge records"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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
    else:
        g = inputs.chung_lu_1m()
    m = g.m

    ctx = gd.Context(device, smem_table_max=args.smem_table, bitmap_max_outdeg=args.bitmap_max,
                     hub_wedges_log2=args.hub_log2, hub_pull=args.hub_pull)
    stream = torch.cuda.Stream(device=device)
    rp = torch.from_numpy(g.row_ptr).to(device)
    ci = torch.from_numpy(g.col_idx).to(device)
    out = None if args.global_only else torch.empty((m, 15), dtype=torch.int64, device=device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)
    torch.cuda.synchronize()
    h = ctx.graph(rp, ci, n=g.n, borrow=True, stream=stream.cuda_stream)

    def step():
        if args.global_only:
            return h.count_global()
        return h.count_per_edge(out=out)[1]

    for _ in range(max(3, args.warmup)):
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
    for _ in range(args.steps):
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

    ms = max_over_ranks(total_ms / args.steps, device)
    value = job_rate(m, ws, ms / 1000.0)

    # end to end through the C ABI with pinned host buffers
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    ci_h = torch.from_numpy(g.col_idx).pin_memory()
    out_h = None if args.global_only else torch.empty((m, 15), dtype=torch.int64).pin_memory()
    h2d = 4 * (g.n + 1) + 4 * g.nnz
    d2h = (0 if args.global_only else 8 * 15 * m) + 16 * 15

    def e2e_step():
        gh = gd.gd_create_csr(ctx.handle, g.n, g.nnz, rp_h.data_ptr(), ci_h.data_ptr(), 0, stream.cuda_stream)
        try:
            if args.global_only:
                r = gd.gd_count_global(ctx.handle, gh)
            else:
                r = gd.gd_count_per_edge(ctx.handle, gh, out_h.data_ptr(), 0, True)
        finally:
            gd.gd_destroy_graph(gh)
        return r

    e2e_step()
    e2e_steps = max(2, min(args.steps, 5))
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r = e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if r != glob:
        raise RuntimeError("end-to-end counts differ from the device-resident counts")
    e2e_s = max_over_ranks(e2e_s, device)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # roofline of the dominant kernel family (all its launches in a step)
    peak, peak_kind = load_peaks()
    kern = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1], "ms_total": v[0]} for k, v in prof.items()}
    fam_ms = {f: sum(kern[k]["ms_total"] for k in names if k in kern) / args.steps
              for f, names in KERNEL_FAMILIES.items()}
    dom = max(fam_ms, key=fam_ms.get)
    ab = algorithmic_bytes(g, int(glob[0]), not args.global_only)
    achieved = ab[dom] / (fam_ms[dom] / 1000.0) / 1e9
    traffic = measured_traffic(g.name, dom)
    roof = {"kernel": dom, "kernels": [k for k in KERNEL_FAMILIES[dom] if k in kern], "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_step": ab[dom],
            "ms_per_step": fam_ms[dom], "per": "step (all launches of the family)",
            "launches_per_step": sum(kern[k]["launches"] for k in KERNEL_FAMILIES[dom] if k in kern) // args.steps,
            "other_families": {f: {"ms_per_step": fam_ms[f], "algorithmic_bytes_per_step": ab[f],
                                   "achieved_gbs": ab[f] / (fam_ms[f] / 1000.0) / 1e9 if fam_ms[f] else None}
                               for f in fam_ms if f != dom}}

    nxt = None
    if not args.global_only and not args.no_batch:
        nxt = run_next_measure(gd, torch, ctx, h, g, out)
    batch = None
    if not args.no_batch:
        batch = run_batch_measure(gd, torch, ctx, device, max(2, min(args.steps, 5)))
    serving = None
    if not args.no_serving:
        serving = run_serving_measure(gd)

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(g, args.cpu_seconds)
        cpu = {k: v for k, v in cpu.items() if not k.startswith("_")}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": g.name, "n": g.n, "m": g.m,
                   "mode": "global" if args.global_only else "per-edge (15 columns) + global",
                   "variant": "oriented", "seed": {"chung_lu_1m": 2, "chung_lu_400k": 9, "rmat_22": 3}[args.workload],
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": job_rate(m, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "launches_before_timed": launches0,
        "family_launches_per_step": {f: sum(kern[k]["launches"] for k in names if k in kern) // args.steps
                                     for f, names in KERNEL_FAMILIES.items()},
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk,
        "batch": batch,
        "serving": serving,
        "updates_and_ranking": nxt,
        "kernels": {k: round(v["ms_total"] / args.steps, 3) for k, v in sorted(kern.items(), key=lambda kv: -kv[1]["ms_total"])},
        "kernel_launches_per_step": {k: v["launches"] // args.steps for k, v in kern.items()},
        "source_digest": source_digest(),
        "global_counts": [str(x) for x in glob],
    }
    print(json.dumps(line), flush=True)
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
