"""gd_count_global_static: the entry point for callers that must not allocate
device memory (for example code that runs beside a latency-critical pipeline,
where cudaMalloc could synchronize the device, or a plug-in whose host
framework owns all device memory).  Its results must equal gd_count_global's
on the same graphs, call after call, even though every call reuses the same
static scratch array.

This file is collected last on purpose: if it fails, every other test has
already run.  It passes alone in a fresh process (the first call sets up the
scratch address) and after the other tests."""
import numpy as np
import pytest

from paper_1506_04322_gb300 import gd, inputs

pytestmark = pytest.mark.gpu


def graphs():
    out = [
        inputs.erdos_renyi_small(),
        inputs.barabasi_albert(3000, 3, 8),
        inputs.chung_lu(20_000, 2.2, 60_000, 0.0, 3),
        inputs.from_edges(5001, [(0, i) for i in range(1, 5001)]),
        inputs.from_edges(40, [(i, j) for i in range(40) for j in range(i + 1, 40)]),
        inputs.from_edges(10, []),
        inputs.erdos_renyi(1200, 0.05, 4),
    ]
    for g in out:
        assert g.n <= gd.GD_STATIC_MAX_N and g.nnz <= gd.GD_STATIC_MAX_NNZ, g.name
    return out


def _u128(out_cpu):
    w = out_cpu.view(np.uint64)
    return [int(w[2 * i]) | (int(w[2 * i + 1]) << 64) for i in range(15)]


def test_static_entry_equals_count_global_twice_in_a_row():
    torch = pytest.importorskip("torch")
    with gd.Context(0) as ctx:
        for g in graphs():
            with ctx.graph(g) as h:
                want = h.count_global()                 # the existing entry point
            rp = torch.from_numpy(g.row_ptr).cuda()
            ci = torch.from_numpy(g.col_idx if g.nnz else np.zeros(1, np.int32)).cuda()
            out = torch.empty(30, dtype=torch.int64, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            for _ in range(2):
                out.fill_(-1)
                torch.cuda.synchronize()
                rc = gd.gd_count_global_static(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), out.data_ptr(), stream)
                assert rc == gd.GD_OK, (g.name, rc)
                assert _u128(out.cpu().numpy()) == want, g.name


def test_static_entry_leaves_device_memory_unchanged():
    """What the entry point is for: after a first call on the device (which
    may load the library's device code and with it the static scratch), more
    calls leave the device's free memory exactly as it was."""
    torch = pytest.importorskip("torch")
    g = inputs.chung_lu(20_000, 2.2, 60_000, 0.0, 3)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    out = torch.empty(30, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert gd.gd_count_global_static(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), out.data_ptr(), stream) == gd.GD_OK
    torch.cuda.synchronize()
    want = _u128(out.cpu().numpy())
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        rc = gd.gd_count_global_static(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), out.data_ptr(), stream)
        assert rc == gd.GD_OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert _u128(out.cpu().numpy()) == want


def test_static_entry_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    rp = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(30, dtype=torch.int64, device="cuda")
    rc = gd.gd_count_global_static(gd.GD_STATIC_MAX_N + 1, 0, rp.data_ptr(), rp.data_ptr(), out.data_ptr())
    assert rc == gd.GD_EOVERFLOW
    rc = gd.gd_count_global_static(3, gd.GD_STATIC_MAX_NNZ + 2, rp.data_ptr(), rp.data_ptr(), out.data_ptr())
    assert rc == gd.GD_EOVERFLOW


def test_static_entry_rejects_malformed_csr():
    torch = pytest.importorskip("torch")
    g = inputs.erdos_renyi(60, 0.2, 5)
    out = torch.empty(30, dtype=torch.int64, device="cuda")
    dup = g.col_idx.copy()
    dup[1] = dup[0]                                     # repeated neighbour in row 0
    r = int(np.flatnonzero(np.diff(g.row_ptr) > 0)[1])  # a non-empty row
    loop = g.col_idx.copy()
    loop[g.row_ptr[r]] = r                              # self-loop
    for ci_h in (dup, loop):
        rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr, np.int32)).cuda()
        ci = torch.from_numpy(np.ascontiguousarray(ci_h, np.int32)).cuda()
        rc = gd.gd_count_global_static(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), out.data_ptr())
        assert rc == gd.GD_EINVAL
