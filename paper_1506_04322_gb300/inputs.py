"""Seeded synthetic inputs: graphs in sorted int32 CSR and the workload recipes.

This module holds none of the graphlet arithmetic.  It is the one piece shared by
the CUDA path's tests/bench and by the CPU oracle's tests: both count the same
seeded graphs.  The generators themselves are C (``csrc/gdgen.c``), built into
``libgdgen.so`` next to this file; they give bit-identical graphs on x86-64 and
aarch64 (see the header of that file).

Recipes (the shapes of the paper's workloads, Sec. 5; the real networks are not
available, so these synthetic graphs stand in for them):

* ``erdos_renyi_small``   -- G(n=2000, p=0.005), seed 1 (~10K edges).
* ``chung_lu_1m``         -- Chung-Lu, n=1,000,000, Pareto density exponent 2.1,
  expected degree capped at 50,000, ~10M undirected edges, seed 2 (social-network
  skew, like the paper's soc-/socfb-/tech- graphs).
* ``rmat_22``             -- R-MAT scale 22, edge factor 16, (a,b,c,d) =
  (0.57,0.19,0.19,0.05), random relabelling, seed 3 (~64M edges, hub-heavy).
* ``graph_batch``         -- 20,000 small graphs, n ~ U{20..500}, even i
  Erdos-Renyi with mean degree ~ U[2,12], odd i Barabasi-Albert with m in {1,2,3},
  seed 4+i (the graph-classification collections of Sec. 6).
* ``request_trace``       -- counting requests: Chung-Lu graphs, m_target
  log-uniform on [1e3, 5e6], exponent ~ U[2.0, 2.8], n = max(32, m_target/8),
  cap sqrt(sum w); Poisson arrival times; seed 5.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgdgen.so")
_SRC_PATH = os.path.join(_HERE, "csrc", "gdgen.c")
_lib = None
_lock = threading.Lock()


def build_generators(force: bool = False) -> str:
    """Compile ``csrc/gdgen.c`` into ``libgdgen.so`` (host C, no CUDA)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC_PATH)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, _SRC_PATH, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build_generators()
        lib = ctypes.CDLL(_LIB_PATH)
        vp = ctypes.c_void_p
        lib.gdgen_erdos_renyi.restype = vp
        lib.gdgen_erdos_renyi.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64]
        lib.gdgen_chung_lu.restype = vp
        lib.gdgen_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int64,
                                       ctypes.c_double, ctypes.c_uint64]
        lib.gdgen_rmat.restype = vp
        lib.gdgen_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
        lib.gdgen_barabasi_albert.restype = vp
        lib.gdgen_barabasi_albert.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64]
        lib.gdgen_from_pairs.restype = vp
        lib.gdgen_from_pairs.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp]
        lib.gdgen_n.restype = ctypes.c_int32
        lib.gdgen_n.argtypes = [vp]
        lib.gdgen_nnz.restype = ctypes.c_int64
        lib.gdgen_nnz.argtypes = [vp]
        lib.gdgen_copy.restype = None
        lib.gdgen_copy.argtypes = [vp, vp, vp]
        lib.gdgen_free.restype = None
        lib.gdgen_free.argtypes = [vp]
        lib.gdgen_uniforms.restype = None
        lib.gdgen_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, vp]
        lib.gdgen_log.restype = ctypes.c_double
        lib.gdgen_log.argtypes = [ctypes.c_double]
        lib.gdgen_exp.restype = ctypes.c_double
        lib.gdgen_exp.argtypes = [ctypes.c_double]
        _lib = lib
        return lib


@dataclasses.dataclass
class Graph:
    """Undirected simple graph in CSR: both directions stored, rows ascending."""
    n: int
    row_ptr: np.ndarray   # int32[n+1]
    col_idx: np.ndarray   # int32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edges(self) -> np.ndarray:
        """(m, 2) int32 array of undirected edges (u, v), u < v, in CSR order."""
        rows = np.repeat(np.arange(self.n, dtype=np.int32), self.degrees())
        keep = rows < self.col_idx
        return np.stack([rows[keep], self.col_idx[keep]], axis=1)


def _take(handle, name: str) -> Graph:
    lib = _load()
    if not handle:
        raise ValueError(f"generator {name} failed (bad parameters or out of memory)")
    try:
        n = lib.gdgen_n(handle)
        nnz = lib.gdgen_nnz(handle)
        rp = np.empty(n + 1, dtype=np.int32)
        ci = np.empty(max(nnz, 1), dtype=np.int32)
        lib.gdgen_copy(handle, rp.ctypes.data, ci.ctypes.data)
        return Graph(n=n, row_ptr=rp, col_idx=ci[:nnz].copy(), name=name)
    finally:
        lib.gdgen_free(handle)


def erdos_renyi(n: int, p: float, seed: int) -> Graph:
    return _take(_load().gdgen_erdos_renyi(n, p, seed), f"er(n={n},p={p},seed={seed})")


def chung_lu(n: int, gamma: float, draws: int, cap: float, seed: int) -> Graph:
    """cap <= 0 selects sqrt(sum w)."""
    return _take(_load().gdgen_chung_lu(n, gamma, draws, cap, seed),
                 f"chung_lu(n={n},gamma={gamma},draws={draws},cap={cap},seed={seed})")


def rmat(scale: int, samples: int, a: float, b: float, c: float, seed: int,
         relabel: bool = True) -> Graph:
    return _take(_load().gdgen_rmat(scale, samples, a, b, c, seed, int(relabel)),
                 f"rmat(scale={scale},samples={samples},seed={seed})")


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    return _take(_load().gdgen_barabasi_albert(n, m, seed), f"ba(n={n},m={m},seed={seed})")


def from_edges(n: int, edges) -> Graph:
    """Simple undirected graph on n nodes from any iterable of (u, v) pairs."""
    e = np.asarray(list(edges) if not isinstance(edges, np.ndarray) else edges,
                   dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    h = _load().gdgen_from_pairs(n, e.shape[0], src.ctypes.data, dst.ctypes.data)
    return _take(h, f"pairs(n={n},m={e.shape[0]})")


def uniforms(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().gdgen_uniforms(seed, stream, count, out.ctypes.data)
    return out


# ----------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------

CHUNG_LU_1M_DRAWS = 11_150_000


def erdos_renyi_small(seed: int = 1) -> Graph:
    g = erdos_renyi(2000, 0.005, seed)
    g.name = "erdos_renyi_n2000_p0.005"
    return g


def chung_lu_1m(seed: int = 2) -> Graph:
    g = chung_lu(1_000_000, 2.1, CHUNG_LU_1M_DRAWS, 50_000.0, seed)
    g.name = "chung_lu_n1M_gamma2.1_cap50k"
    return g


def rmat_22(seed: int = 3) -> Graph:
    g = rmat(22, 16 << 22, 0.57, 0.19, 0.19, seed, True)
    g.name = "rmat_scale22_ef16"
    return g


def batch_graph_params(index: int, seed: int = 4):
    """(kind, n, param) of graph `index` of the batch recipe."""
    u = uniforms(seed + index, 7, 3)
    n = 20 + int(u[0] * 481)                      # U{20..500}
    if index % 2 == 0:
        dbar = 2.0 + 10.0 * u[1]                  # U[2,12]
        return "er", n, dbar / (n - 1)
    return "ba", n, 1 + int(u[1] * 3)             # U{1,2,3}


def batch_graph(index: int, seed: int = 4) -> Graph:
    kind, n, prm = batch_graph_params(index, seed)
    if kind == "er":
        return erdos_renyi(n, prm, seed + index)
    return barabasi_albert(n, prm, seed + index)


def graph_batch(count: int = 20_000, seed: int = 4) -> list[Graph]:
    return [batch_graph(i, seed) for i in range(count)]


@dataclasses.dataclass
class PackedBatch:
    """Many graphs in one CSR: node ids are global, graph g owns nodes
    graph_node_ptr[g] .. graph_node_ptr[g+1]-1 and never links outside them."""
    num_graphs: int
    graph_node_ptr: np.ndarray   # int32[G+1]
    row_ptr: np.ndarray          # int32[N+1]
    col_idx: np.ndarray          # int32[nnz]


def pack(graphs: list[Graph]) -> PackedBatch:
    gnp = np.zeros(len(graphs) + 1, dtype=np.int64)
    gnp[1:] = np.cumsum([g.n for g in graphs])
    nnz = np.zeros(len(graphs) + 1, dtype=np.int64)
    nnz[1:] = np.cumsum([g.nnz for g in graphs])
    if gnp[-1] >= 2**31 - 1 or nnz[-1] >= 2**31 - 1:
        raise OverflowError("packed batch exceeds int32 ids")
    rp = np.empty(gnp[-1] + 1, dtype=np.int32)
    ci = np.empty(nnz[-1], dtype=np.int32)
    for i, g in enumerate(graphs):
        rp[gnp[i]:gnp[i + 1]] = g.row_ptr[:-1] + nnz[i]
        ci[nnz[i]:nnz[i + 1]] = g.col_idx + gnp[i]
    rp[-1] = nnz[-1]
    return PackedBatch(len(graphs), gnp.astype(np.int32), rp, ci)


@dataclasses.dataclass
class Request:
    index: int
    arrival_s: float
    gamma: float
    m_target: int
    n: int
    seed: int

    def graph(self) -> Graph:
        g = chung_lu(self.n, self.gamma, self.m_target, 0.0, self.seed)
        g.name = f"request{self.index}"
        return g


def request_trace(count: int = 5000, rate_per_s: float = 100.0, seed: int = 5,
                  m_lo: float = 1e3, m_hi: float = 5e6) -> list[Request]:
    """Requests with Poisson arrivals at `rate_per_s`; sizes log-uniform."""
    lib = _load()
    u = uniforms(seed, 11, 3 * count)
    lo, hi = lib.gdgen_log(m_lo), lib.gdgen_log(m_hi)
    t = 0.0
    out = []
    for i in range(count):
        gap = -lib.gdgen_log(1.0 - u[3 * i]) / rate_per_s
        t += gap
        m_t = int(lib.gdgen_exp(lo + (hi - lo) * u[3 * i + 1]))
        gamma = 2.0 + 0.8 * u[3 * i + 2]
        n = max(32, m_t // 8)
        out.append(Request(i, t, gamma, m_t, n, seed * 1_000_003 + i))
    return out
