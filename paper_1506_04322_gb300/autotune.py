"""Autotuner cache: options found by gd_autotune, keyed by GPU, mode and a
summary of the graph's degree histogram (log2 buckets), stored as JSON.

The paper's auto-optimizer (Sec. 5.2) picks data structures by graph density;
here the knobs are libgd's kernel cut-overs (shared-memory wedge table size,
bitmap out-degree limit, hub wedge threshold) and, for batches of small
graphs, the batched kernel's CTA size.  Counts are exact under every option
set, so a stale cache entry can only cost time, never change a result.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import gd


def degree_signature(g) -> str:
    """n, m and the degree histogram in log2 buckets, coarsened to 1 significant
    digit, so that graphs of the same family and size share an entry."""
    d = np.diff(np.asarray(g.row_ptr, dtype=np.int64))
    buckets = np.zeros(33, dtype=np.int64)
    if d.size:
        b = np.where(d > 0, np.floor(np.log2(np.maximum(d, 1))).astype(np.int64) + 1, 0)
        buckets = np.bincount(b, minlength=33)

    def coarse(x: int) -> str:
        return "0" if x == 0 else f"{float(f'{x:.1g}'):g}"
    return f"n{coarse(g.n)}_m{coarse(int(g.row_ptr[-1]) // 2)}_h" + ".".join(coarse(int(x)) for x in buckets)


def _gpu_name(device: int) -> str:
    try:
        import torch
        return torch.cuda.get_device_name(device).replace(" ", "_")
    except Exception:
        return f"cuda{device}"


def tuned_options(ctx: "gd.Context", graph_handle: "gd.Graph", g, per_edge: bool = False,
                  cache_path: str | None = None, max_trials: int = 24, device: int = 0) -> dict:
    """Options for this graph: from the cache, else by gd_autotune (and then
    cached).  The context's options are set either way."""
    path = cache_path or os.environ.get("GD_TUNE_CACHE")
    key = f"{_gpu_name(device)}|{'per_edge' if per_edge else 'global'}|{degree_signature(g)}"
    cache = {}
    if path and os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    if key in cache:
        o = gd.gd_default_options()
        o.variant = ctx.variant
        for k, v in cache[key]["options"].items():
            setattr(o, k, v)
        ctx.set_options(o)
        return dict(cache[key], cached=True)
    res = graph_handle.autotune(per_edge=per_edge, max_trials=max_trials)
    entry = {"options": {k: res[k] for k in ("smem_table_max", "bitmap_max_outdeg", "hub_wedges_log2",
                                             "medium_cluster_log2")},
             "best_ms": res["best_ms"], "default_ms": res["default_ms"], "trials": res["trials"]}
    if path:
        cache[key] = entry
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return dict(entry, cached=False)


def batch_signature(graph_node_ptr, row_ptr) -> str:
    """Graph count, node and edge totals and the node-count histogram (log2
    buckets), coarsened like degree_signature."""
    gnp = np.asarray(graph_node_ptr, dtype=np.int64)
    sizes = np.diff(gnp)
    b = np.bincount(np.floor(np.log2(np.maximum(sizes, 1))).astype(np.int64), minlength=17) if sizes.size else []

    def coarse(x: int) -> str:
        return "0" if x == 0 else f"{float(f'{x:.1g}'):g}"
    nnz = int(np.asarray(row_ptr)[-1])
    return f"G{coarse(len(sizes))}_N{coarse(int(gnp[-1]))}_E{coarse(nnz // 2)}_h" + ".".join(coarse(int(x)) for x in b)


def tuned_batch_options(ctx: "gd.Context", batch, cache_path: str | None = None, device: int = 0) -> dict:
    """batch_threads for this kind of batch (host-side packed arrays): from
    the cache, else by gd_autotune_batch (and then cached)."""
    path = cache_path or os.environ.get("GD_TUNE_CACHE")
    key = f"{_gpu_name(device)}|batch|{batch_signature(batch.graph_node_ptr, batch.row_ptr)}"
    cache = {}
    if path and os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    if key in cache:
        o = ctx.options()
        o.batch_threads = cache[key]["options"]["batch_threads"]
        ctx.set_options(o)
        return dict(cache[key], cached=True)
    res = ctx.autotune_batch(batch)
    entry = {"options": {"batch_threads": res["batch_threads"]}, "best_ms": res["best_ms"],
             "default_ms": res["default_ms"], "trials": res["trials"]}
    if path:
        cache[key] = entry
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return dict(entry, cached=False)
