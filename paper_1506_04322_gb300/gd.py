"""Python binding of libgd (include/gd.h): argument marshalling only.

Every count runs in the CUDA kernels of ``libgd.so``; nothing here computes
graphlet counts.  If the library is not built, every call raises -- there is no
CPU fallback.

Two layers:

* functions with the C names (``gd_init``, ``gd_create_csr``, ``gd_count_global``,
  ``gd_count_per_edge``, ``gd_count_batch``, ...) taking handles and raw pointers;
* ``Context`` / ``Graph`` wrappers that accept numpy arrays (host memory) or torch
  tensors (device memory, via ``data_ptr()``) and torch streams.

Counts come back in Table 1 order [g31 g32 g33 g34 g41 ... g4_10 g4_11].
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgd.so")
HEADER = os.path.join(HERE, "..", "include", "gd.h")

GRAPHLETS = ["g31", "g32", "g33", "g34", "g41", "g42", "g43", "g44", "g45", "g46",
             "g47", "g48", "g49", "g4_10", "g4_11"]

GD_OK, GD_EINVAL, GD_ENOMEM, GD_ECUDA, GD_EAGAIN, GD_ETIMEDOUT, GD_EOVERFLOW, GD_ENOTIMPL, GD_EARITH = range(9)
STATUS_NAMES = {0: "GD_OK", 1: "GD_EINVAL", 2: "GD_ENOMEM", 3: "GD_ECUDA", 4: "GD_EAGAIN",
                5: "GD_ETIMEDOUT", 6: "GD_EOVERFLOW", 7: "GD_ENOTIMPL", 8: "GD_EARITH"}
GD_DEVICE_PTRS, GD_VALIDATE, GD_BORROW = 1, 2, 4
GD_OUT_DEVICE = 1
GD_CAPTURE = 8
GD_VARIANT_AUTO, GD_VARIANT_LITERAL, GD_VARIANT_ORIENTED = 0, 1, 2
GD_PULL_AUTO, GD_PULL_NEVER, GD_PULL_ALWAYS = 0, 1, 2


class GDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class gd_u128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]


class gd_stage_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("ms_total", ctypes.c_double), ("launches", ctypes.c_int64)]


class gd_request_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("mode", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gd_req_stats(ctypes.Structure):
    _fields_ = [("submit_ms", ctypes.c_double), ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double),
                ("footprint", ctypes.c_size_t), ("slot", ctypes.c_int32), ("batched", ctypes.c_int32)]


class gd_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("smem_table_max", ctypes.c_int32),
                ("bitmap_max_outdeg", ctypes.c_int32), ("hub_wedges_log2", ctypes.c_int32),
                ("hub_pull", ctypes.c_int32), ("batch_threads", ctypes.c_int32),
                ("medium_cluster_log2", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class gd_tune_result(ctypes.Structure):
    _fields_ = [("best", gd_options), ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("trials", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load():
    """Load libgd.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgd.so is not built; run paper_1506_04322_gb300.build.build() "
                               "(nvcc for sm_103a) -- there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "gd_default_options": (None, [vp]),
            "gd_init": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, sz, vp]),
            "gd_destroy": (None, [vp]),
            "gd_last_error": (ctypes.c_char_p, [vp]),
            "gd_create_csr": (ctypes.c_int, [vp, i32, i64, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)]),
            "gd_graph_info": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i64)]),
            "gd_graph_footprint": (ctypes.c_int, [vp, ctypes.POINTER(sz)]),
            "gd_destroy_graph": (None, [vp]),
            "gd_count_global": (ctypes.c_int, [vp, vp]),
            "gd_count_per_edge": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
            "gd_count_batch": (ctypes.c_int, [vp, i32, vp, vp, vp, ctypes.c_int, vp]),
            "gd_count_batch_gather": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, ctypes.c_int, vp]),
            "gd_profile_begin": (ctypes.c_int, [vp]),
            "gd_profile_end": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32)]),
            "gd_kernel_launches": (i64, [vp]),
            "gd_pool_release": (ctypes.c_int, [vp]),
            "gd_count_global_static": (ctypes.c_int, [i32, i64, vp, vp, vp, vp]),
            "gd_serve_start": (ctypes.c_int, [vp, i32, sz]),
            "gd_submit": (ctypes.c_int, [vp, vp, ctypes.POINTER(ctypes.c_uint64)]),
            "gd_poll": (ctypes.c_int, [vp, ctypes.c_uint64, vp, vp]),
            "gd_wait": (ctypes.c_int, [vp, ctypes.c_uint64, i32]),
            "gd_serve_stats": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
            "gd_serve_stop": (ctypes.c_int, [vp]),
            "gd_footprint_estimate": (ctypes.c_int, [vp, i32, i64, ctypes.c_int, ctypes.POINTER(sz)]),
            "gd_autotune": (ctypes.c_int, [vp, ctypes.c_int, i32, vp]),
            "gd_autotune_batch": (ctypes.c_int, [vp, i32, vp, vp, vp, ctypes.c_int, vp, vp]),
            "gd_set_options": (ctypes.c_int, [vp, vp]),
            "gd_get_options": (ctypes.c_int, [vp, vp]),
            "gd_topk": (ctypes.c_int, [vp, vp, i64, i64, ctypes.c_int, i64, vp, vp, vp]),
            "gd_toggle_delta": (ctypes.c_int, [vp, i32, i32, vp, vp, ctypes.POINTER(ctypes.c_int)]),
            "gd_node_sums": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]),
            "gd_gfd": (ctypes.c_int, [i64, i64, vp, vp]),
            "gd_gfd_batch": (ctypes.c_int, [vp, i32, vp, vp, vp, ctypes.c_int, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def declared_symbols() -> list[str]:
    """Function names declared in include/gd.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gd_[a-z0-9_]+)\s*\(", text)))


# ---------------------------------------------------------------------------
# C-named thin wrappers
# ---------------------------------------------------------------------------

def _u128_list(arr) -> list[int]:
    return [int(x.lo) | (int(x.hi) << 64) for x in arr]


def gd_default_options() -> gd_options:
    o = gd_options()
    load().gd_default_options(ctypes.byref(o))
    return o


def gd_init(device: int = 0, hbm_budget_bytes: int = 0, options: gd_options | None = None):
    h = ctypes.c_void_p()
    rc = load().gd_init(ctypes.byref(h), device, hbm_budget_bytes,
                        ctypes.byref(options) if options is not None else None)
    if rc:
        raise GDError(rc, "gd_init failed")
    return h


def gd_destroy(ctx) -> None:
    load().gd_destroy(ctx)


def gd_last_error(ctx) -> str:
    s = load().gd_last_error(ctx)
    return s.decode() if s else ""


def _check(ctx, rc, what):
    if rc:
        raise GDError(rc, f"{what}: {gd_last_error(ctx)}")


def gd_create_csr(ctx, n: int, nnz: int, row_ptr: int, col_idx: int, flags: int = 0, stream: int = 0):
    h = ctypes.c_void_p()
    rc = load().gd_create_csr(ctx, n, nnz, row_ptr, col_idx, flags, stream or None, ctypes.byref(h))
    _check(ctx, rc, "gd_create_csr")
    return h


def gd_destroy_graph(graph) -> None:
    load().gd_destroy_graph(graph)


def gd_graph_info(graph) -> tuple[int, int]:
    n, m = ctypes.c_int32(), ctypes.c_int64()
    load().gd_graph_info(graph, ctypes.byref(n), ctypes.byref(m))
    return n.value, m.value


def gd_graph_footprint(graph) -> int:
    b = ctypes.c_size_t()
    load().gd_graph_footprint(graph, ctypes.byref(b))
    return b.value


def gd_count_global(ctx, graph) -> list[int]:
    out = (gd_u128 * 15)()
    _check(ctx, load().gd_count_global(graph, out), "gd_count_global")
    return _u128_list(out)


def gd_count_per_edge(ctx, graph, out_ptr: int, out_flags: int = 0, want_global: bool = True):
    glob = (gd_u128 * 15)() if want_global else None
    _check(ctx, load().gd_count_per_edge(graph, out_ptr, out_flags, glob), "gd_count_per_edge")
    return _u128_list(glob) if want_global else None


def gd_count_batch(ctx, num_graphs: int, graph_node_ptr: int, row_ptr: int, col_idx: int,
                   flags: int, out_ptr: int) -> None:
    _check(ctx, load().gd_count_batch(ctx, num_graphs, graph_node_ptr, row_ptr, col_idx, flags, out_ptr),
           "gd_count_batch")


def gd_count_batch_gather(ctx, num_graphs: int, row_ptrs: int, col_idxs: int, num_nodes: int, num_slots: int,
                          flags: int, out_ptr: int) -> None:
    """row_ptrs / col_idxs: device arrays of device pointers; num_nodes
    (int32) / num_slots (int64): host arrays; out: device."""
    _check(ctx, load().gd_count_batch_gather(ctx, num_graphs, row_ptrs, col_idxs, num_nodes, num_slots, flags,
                                             out_ptr), "gd_count_batch_gather")


def gd_profile_begin(ctx) -> None:
    _check(ctx, load().gd_profile_begin(ctx), "gd_profile_begin")


def gd_profile_end(ctx) -> dict:
    """{kernel name: (total ms, launches)} collected since gd_profile_begin."""
    num = ctypes.c_int32()
    buf = (gd_stage_stat * 64)()
    _check(ctx, load().gd_profile_end(ctx, buf, 64, ctypes.byref(num)), "gd_profile_end")
    return {buf[i].name.decode(): (buf[i].ms_total, buf[i].launches) for i in range(min(num.value, 64))}


def gd_kernel_launches(ctx) -> int:
    return int(load().gd_kernel_launches(ctx))


def gd_pool_release(ctx) -> None:
    _check(ctx, load().gd_pool_release(ctx), "gd_pool_release")


GD_STATIC_MAX_N = 32768
GD_STATIC_MAX_NNZ = 262144


def gd_count_global_static(n: int, nnz: int, row_ptr: int, col_idx: int, out: int, stream: int = 0) -> int:
    """Global counts without allocating (device pointers in and out; see
    include/gd.h).  Returns the gd_status code."""
    return int(load().gd_count_global_static(n, nnz, row_ptr, col_idx, out, stream or None))


def gd_toggle_delta(ctx, graph, u: int, v: int):
    """(gain, loss, was_edge) of toggling the pair {u, v}: counts after the
    toggle = counts + gain - loss."""
    gain, loss = (gd_u128 * 15)(), (gd_u128 * 15)()
    was = ctypes.c_int()
    _check(ctx, load().gd_toggle_delta(graph, u, v, gain, loss, ctypes.byref(was)), "gd_toggle_delta")
    return _u128_list(gain), _u128_list(loss), bool(was.value)


def gd_topk(ctx, values_ptr: int, count: int, stride: int, k: int, device: bool, stream: int = 0):
    """(indices int64[k], values uint64[k]) of the k largest values[i * stride],
    value descending, ties by ascending index."""
    idx = np.zeros(max(k, 1), dtype=np.int64)
    val = np.zeros(max(k, 1), dtype=np.uint64)
    _check(ctx, load().gd_topk(ctx, values_ptr, count, stride, GD_DEVICE_PTRS if device else 0, k,
                               idx.ctypes.data, val.ctypes.data, stream or None), "gd_topk")
    return idx[:k], val[:k]


def gd_node_sums(ctx, graph, per_edge_ptr: int, device: bool, column: int, out_ptr: int, out_device: bool) -> None:
    _check(ctx, load().gd_node_sums(graph, per_edge_ptr, GD_DEVICE_PTRS if device else 0, column, out_ptr,
                                    GD_OUT_DEVICE if out_device else 0), "gd_node_sums")


def gd_gfd(n: int, m: int, counts) -> np.ndarray:
    """17 normalised frequencies (k = 2, 3, 4) from the 15 exact counts."""
    c = (gd_u128 * 15)()
    for i, x in enumerate(counts):
        c[i].lo = int(x) & (2**64 - 1)
        c[i].hi = int(x) >> 64
    out = np.zeros(17, dtype=np.float64)
    rc = load().gd_gfd(n, m, c, out.ctypes.data)
    if rc != GD_OK:
        raise GDError(rc, "gd_gfd: invalid arguments")
    return out


def gd_gfd_batch(ctx, num_graphs: int, graph_node_ptr: int, row_ptr: int, counts: int, out: int,
                 stream: int = 0) -> None:
    _check(ctx, load().gd_gfd_batch(ctx, num_graphs, graph_node_ptr, row_ptr, counts, GD_DEVICE_PTRS, out,
                                    stream or None), "gd_gfd_batch")


def gd_autotune_batch(ctx, num_graphs: int, graph_node_ptr: int, row_ptr: int, col_idx: int, flags: int,
                      out_ptr: int) -> dict:
    r = gd_tune_result()
    _check(ctx, load().gd_autotune_batch(ctx, num_graphs, graph_node_ptr, row_ptr, col_idx, flags, out_ptr,
                                         ctypes.byref(r)), "gd_autotune_batch")
    return {"batch_threads": r.best.batch_threads, "best_ms": r.best_ms, "default_ms": r.default_ms,
            "trials": r.trials}


def gd_autotune(ctx, graph, per_edge: bool = False, max_trials: int = 24) -> dict:
    r = gd_tune_result()
    _check(ctx, load().gd_autotune(graph, int(per_edge), max_trials, ctypes.byref(r)), "gd_autotune")
    b = r.best
    return {"smem_table_max": b.smem_table_max, "bitmap_max_outdeg": b.bitmap_max_outdeg,
            "hub_wedges_log2": b.hub_wedges_log2, "medium_cluster_log2": b.medium_cluster_log2,
            "best_ms": r.best_ms, "default_ms": r.default_ms,
            "trials": r.trials}


def gd_serve_start(ctx, slots: int = 4, hbm_budget_bytes: int = 0) -> None:
    _check(ctx, load().gd_serve_start(ctx, slots, hbm_budget_bytes), "gd_serve_start")


def gd_submit(ctx, n: int, nnz: int, row_ptr: int, col_idx: int) -> int:
    d = gd_request_desc(n, nnz, row_ptr, col_idx, 0, 0)
    rid = ctypes.c_uint64()
    rc = load().gd_submit(ctx, ctypes.byref(d), ctypes.byref(rid))
    if rc:
        raise GDError(rc, "gd_submit")
    return rid.value


def gd_poll(ctx, rid: int):
    """(status, counts or None, stats dict or None); status GD_EAGAIN while running."""
    out = (gd_u128 * 15)()
    st = gd_req_stats()
    rc = load().gd_poll(ctx, rid, out, ctypes.byref(st))
    if rc == GD_EAGAIN:
        return rc, None, None
    stats = {"submit_ms": st.submit_ms, "start_ms": st.start_ms, "end_ms": st.end_ms,
             "footprint": st.footprint, "slot": st.slot, "batched": st.batched}
    return rc, (_u128_list(out) if rc == GD_OK else None), stats


def gd_wait(ctx, rid: int, timeout_ms: int = -1) -> int:
    return int(load().gd_wait(ctx, rid, timeout_ms))


def gd_serve_stats(ctx) -> dict:
    q, r, b, bl, sl = (ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_int64(), ctypes.c_int64())
    _check(ctx, load().gd_serve_stats(ctx, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b), ctypes.byref(bl),
                                      ctypes.byref(sl)), "gd_serve_stats")
    return {"queued": q.value, "running": r.value, "inflight_bytes": b.value,
            "batched_launches": bl.value, "single_launches": sl.value}


def gd_serve_stop(ctx) -> None:
    load().gd_serve_stop(ctx)


def gd_footprint_estimate(ctx, n: int, nnz: int, per_edge: bool = False) -> int:
    b = ctypes.c_size_t()
    _check(ctx, load().gd_footprint_estimate(ctx, n, nnz, int(per_edge), ctypes.byref(b)), "gd_footprint_estimate")
    return b.value


# ---------------------------------------------------------------------------
# object layer
# ---------------------------------------------------------------------------

def _ptr(a):
    """(pointer, is_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be contiguous")
        return a.ctypes.data, False
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), bool(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class Context:
    """A libgd context on one GPU."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, variant: int = GD_VARIANT_AUTO,
                 smem_table_max: int | None = None, bitmap_max_outdeg: int | None = None,
                 hub_wedges_log2: int | None = None, hub_pull: int | None = None,
                 medium_cluster_log2: int | None = None):
        o = gd_default_options()
        o.variant = variant
        if medium_cluster_log2 is not None:
            o.medium_cluster_log2 = medium_cluster_log2
        if hub_pull is not None:
            o.hub_pull = hub_pull
        if smem_table_max:
            o.smem_table_max = smem_table_max
        if bitmap_max_outdeg:
            o.bitmap_max_outdeg = bitmap_max_outdeg
        if hub_wedges_log2:
            o.hub_wedges_log2 = hub_wedges_log2
        self.handle = gd_init(device, hbm_budget_bytes, o)
        self.variant = variant
        self._graphs = []

    def close(self):
        if self.handle:
            gd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def last_error(self) -> str:
        return gd_last_error(self.handle)

    def set_options(self, o: gd_options) -> None:
        _check(self.handle, load().gd_set_options(self.handle, ctypes.byref(o)), "gd_set_options")

    def options(self) -> gd_options:
        o = gd_options()
        _check(self.handle, load().gd_get_options(self.handle, ctypes.byref(o)), "gd_get_options")
        return o

    def profile_begin(self) -> None:
        gd_profile_begin(self.handle)

    def profile_end(self) -> dict:
        return gd_profile_end(self.handle)

    def kernel_launches(self) -> int:
        return gd_kernel_launches(self.handle)

    # request loop
    def serve_start(self, slots: int = 4, hbm_budget_bytes: int = 0) -> None:
        gd_serve_start(self.handle, slots, hbm_budget_bytes)

    def submit(self, g) -> int:
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(g.col_idx if g.nnz else np.zeros(1, np.int32), dtype=np.int32)
        return gd_submit(self.handle, g.n, int(g.row_ptr[-1]), rp.ctypes.data, ci.ctypes.data)

    def poll(self, rid: int):
        return gd_poll(self.handle, rid)

    def wait(self, rid: int, timeout_ms: int = -1) -> int:
        return gd_wait(self.handle, rid, timeout_ms)

    def serve_stats(self) -> dict:
        return gd_serve_stats(self.handle)

    def serve_stop(self) -> None:
        gd_serve_stop(self.handle)

    def footprint_estimate(self, n: int, nnz: int, per_edge: bool = False) -> int:
        return gd_footprint_estimate(self.handle, n, nnz, per_edge)

    def topk(self, values, k: int, column: int | None = None):
        """The k largest entries (indices, values), value descending and ties
        by ascending index.  values: uint64 vector, or an [rows, 15] per-edge
        matrix with `column` chosen (numpy on the host or torch on the GPU)."""
        ptr, dev = _ptr(values)
        if column is not None:
            rows, cols = values.shape
            return gd_topk(self.handle, ptr + 8 * column, rows, cols, k, dev)
        return gd_topk(self.handle, ptr, int(values.shape[0]), 1, k, dev)

    def graph(self, row_ptr, col_idx=None, n: int | None = None, validate: bool = False,
              borrow: bool = False, stream: int | None = None) -> "Graph":
        """Upload a CSR graph: numpy arrays, torch tensors, or an object with
        ``row_ptr``/``col_idx``/``n`` attributes (inputs.Graph)."""
        if col_idx is None:
            g = row_ptr
            row_ptr, col_idx, n = g.row_ptr, g.col_idx, g.n
        if n is None:
            n = int(row_ptr.shape[0]) - 1
        nnz = int(col_idx.shape[0])
        if isinstance(row_ptr, np.ndarray):
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
            col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
            if col_idx.size == 0:
                col_idx = np.zeros(1, dtype=np.int32)
        keep = [row_ptr, col_idx]
        rp, dev = _ptr(row_ptr)
        ci, dev2 = _ptr(col_idx)
        if dev != dev2:
            raise ValueError("row_ptr and col_idx must both be on the host or both on the device")
        flags = (GD_DEVICE_PTRS if dev else 0) | (GD_VALIDATE if validate else 0) | (GD_BORROW if borrow else 0)
        st = _torch_stream() if stream is None else stream
        h = gd_create_csr(self.handle, n, nnz, rp, ci, flags, st)
        gr = Graph(self, h, keep if borrow else None)
        return gr

    def count_batch(self, batch, out=None, validate: bool = False, device_out: bool = False,
                    capture: bool = False):
        """Per-graph global counts of a packed batch (inputs.PackedBatch or
        arrays/tensors graph_node_ptr, row_ptr, col_idx).  Returns a uint64
        array [G, 15] (numpy, or the given/allocated torch tensor)."""
        gnp, rp, ci = batch.graph_node_ptr, batch.row_ptr, batch.col_idx
        G = int(gnp.shape[0]) - 1
        pg, dev = _ptr(gnp)
        pr, _ = _ptr(rp)
        pc, _ = _ptr(ci if ci.shape[0] > 0 else (np.zeros(1, np.int32) if not dev else ci))
        flags = (GD_DEVICE_PTRS if dev else 0) | (GD_VALIDATE if validate else 0)
        if out is None:
            if device_out:
                import torch
                out = torch.empty((max(G, 1), 15), dtype=torch.int64, device="cuda")
            else:
                out = np.zeros((max(G, 1), 15), dtype=np.uint64)
        po, odev = _ptr(out)
        if odev:
            flags |= GD_OUT_DEVICE
        if capture:
            flags |= GD_CAPTURE
        gd_count_batch(self.handle, G, pg, pr, pc, flags, po)
        return out[:G]

    def autotune_batch(self, batch, out=None) -> dict:
        """gd_autotune_batch on a packed batch (the batch_threads option)."""
        gnp, rp, ci = batch.graph_node_ptr, batch.row_ptr, batch.col_idx
        G = int(gnp.shape[0]) - 1
        pg, dev = _ptr(gnp)
        pr, _ = _ptr(rp)
        pc, _ = _ptr(ci if ci.shape[0] > 0 else (np.zeros(1, np.int32) if not dev else ci))
        if out is None:
            out = np.zeros((max(G, 1), 15), dtype=np.uint64)
        po, odev = _ptr(out)
        flags = (GD_DEVICE_PTRS if dev else 0) | (GD_OUT_DEVICE if odev else 0)
        return gd_autotune_batch(self.handle, G, pg, pr, pc, flags, po)

    def count_batch_gather(self, graphs, out=None, capture: bool = False):
        """Per-graph global counts of graphs held as separate device CSRs:
        `graphs` is a list of (row_ptr, col_idx) torch int32 CUDA tensors.
        Returns a torch int64 tensor [G, 15] (uint64 bit patterns)."""
        import torch
        G = len(graphs)
        dev = graphs[0][0].device if G else torch.device("cuda")
        rps = torch.tensor([r.data_ptr() for r, _ in graphs], dtype=torch.int64, device=dev)
        cis = torch.tensor([c.data_ptr() for _, c in graphs], dtype=torch.int64, device=dev)
        nn = np.array([r.shape[0] - 1 for r, _ in graphs], dtype=np.int32)
        ns = np.array([c.shape[0] for _, c in graphs], dtype=np.int64)
        if out is None:
            out = torch.empty((max(G, 1), 15), dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        gd_count_batch_gather(self.handle, G, rps.data_ptr(), cis.data_ptr(), nn.ctypes.data, ns.ctypes.data,
                              GD_CAPTURE if capture else 0, out.data_ptr())
        self._keep = (rps, cis)
        return out[:G]


class Graph:
    def __init__(self, ctx: Context, handle, keep):
        self.ctx = ctx
        self.handle = handle
        self._keep = keep
        self.n, self.m = gd_graph_info(handle)

    def close(self):
        if self.handle and self.ctx.handle:
            gd_destroy_graph(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def footprint(self) -> int:
        return gd_graph_footprint(self.handle)

    def autotune(self, per_edge: bool = False, max_trials: int = 24) -> dict:
        """Time option sets on this graph; the fastest become the context's."""
        return gd_autotune(self.ctx.handle, self.handle, per_edge, max_trials)

    def count_global(self) -> list[int]:
        return gd_count_global(self.ctx.handle, self.handle)

    def toggle_delta(self, u: int, v: int):
        """(gain, loss, was_edge) of inserting or deleting the pair {u, v}."""
        return gd_toggle_delta(self.ctx.handle, self.handle, u, v)

    def node_sums(self, per_edge, column: int, out=None):
        """Per node v, the sum of column `column` of the per-edge matrix over
        the edges at v (numpy or torch CUDA in and out)."""
        pp, pdev = _ptr(per_edge)
        if out is None:
            out = np.zeros(max(self.n, 1), dtype=np.uint64)
        po, odev = _ptr(out)
        gd_node_sums(self.ctx.handle, self.handle, pp, pdev, column, po, odev)
        return out[:self.n]

    def count_per_edge(self, out=None, want_global: bool = True):
        """uint64 [m, 15] per-edge counts (numpy on the host, or into the given
        torch CUDA tensor of shape [m, 15], dtype int64/uint64 bits).
        Returns (per_edge, global_counts)."""
        if out is None:
            out = np.zeros((max(self.m, 1), 15), dtype=np.uint64)
        po, dev = _ptr(out)
        g = gd_count_per_edge(self.ctx.handle, self.handle, po, GD_OUT_DEVICE if dev else 0, want_global)
        return out[:self.m], g
