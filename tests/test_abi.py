"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/gd.h declares.  No compute calls (no GPU)."""
import ctypes
import os
import subprocess

import pytest

from paper_1506_04322_gb300 import build, gd, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(f"nvcc unavailable: {e}")
    return gd.load()


def test_header_declares_the_boundary():
    names = set(gd.declared_symbols())
    for required in ("gd_init", "gd_create_csr", "gd_count_global", "gd_count_per_edge",
                     "gd_count_batch", "gd_destroy_graph", "gd_destroy", "gd_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", gd.LIB_PATH], capture_output=True, text=True)
    exported = {line.split()[-1] for line in out.stdout.splitlines() if line.strip()}
    for name in gd.declared_symbols():
        assert name in exported, name
        assert hasattr(lib, name)


def test_options_layout_and_defaults(lib):
    o = gd.gd_default_options()
    assert o.variant == gd.GD_VARIANT_AUTO
    assert o.smem_table_max >= 256 and (o.smem_table_max & (o.smem_table_max - 1)) == 0
    assert ctypes.sizeof(gd.gd_options) == 48
    assert o.bitmap_max_outdeg == 1024 and o.hub_wedges_log2 == 17
    assert o.hub_pull == gd.GD_PULL_AUTO


def test_generators_are_deterministic_and_simple():
    a = inputs.chung_lu(5000, 2.1, 20000, 500.0, 9)
    b = inputs.chung_lu(5000, 2.1, 20000, 500.0, 9)
    assert (a.row_ptr == b.row_ptr).all() and (a.col_idx == b.col_idx).all()
    for g in (a, inputs.rmat(12, 1 << 15, 0.57, 0.19, 0.19, 3), inputs.barabasi_albert(500, 3, 1),
              inputs.erdos_renyi(300, 0.05, 2)):
        rp, ci = g.row_ptr, g.col_idx
        assert rp[0] == 0 and rp[-1] == len(ci)
        for u in range(g.n):
            row = ci[rp[u]:rp[u + 1]]
            assert (row[1:] > row[:-1]).all() and (row != u).all()
        e = g.edges()
        back = {(int(v), int(u)) for u, v in e}
        assert len(back) == g.m


def test_batch_packing_offsets():
    gs = [inputs.batch_graph(i) for i in range(6)]
    b = inputs.pack(gs)
    assert b.graph_node_ptr[-1] == sum(g.n for g in gs)
    assert b.row_ptr[-1] == sum(g.nnz for g in gs)
