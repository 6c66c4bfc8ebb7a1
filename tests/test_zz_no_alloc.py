"""The allocation-free COO SpMV entry point (gko_spmv_coo_noalloc).

It serves callers that cannot allocate device memory while they run (graph
capture with a fixed footprint, real-time loops, memory owned by another
allocator); its scratch is a fixed array inside the library.  These tests
call it through the C ABI on two calls in a row and compare its output
element by element with the oracle's compensated (Dot2) product, within the
tolerance every SpMV test uses: |y - y_ref| <= 1e-12 * (|alpha| |A| |x| +
|beta| |y|) per entry; the handle-based COO SpMV (gko_spmv) is held to the
same reference on the same inputs.
The file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def _coo_on_device(gko, A, dev):
    import torch
    M = gko.Matrix(A)
    M.convert("coo")
    c = M.export("coo")
    return M, [torch.from_numpy(np.ascontiguousarray(c[k])).to(dev) for k in ("row", "col", "val")]


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.75, 1.25)])
def test_no_alloc_matches_handle_spmv_twice(gko, dev, orc, alpha, beta):
    import torch
    # several tiles, rows crossing tiles, a ragged last tile (nnz not a
    # multiple of 4), empty rows
    A = syn.powerlaw(60000, 20.0, 1.5, 8000, seed=91)
    A = dict(A)
    keep = len(A["val"]) - 3
    while keep % 4 == 0:
        keep -= 1
    rows = np.repeat(np.arange(A["n_rows"]), np.diff(A["row_ptr"]))[:keep]
    A["row_ptr"] = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=A["n_rows"]))]).astype(np.int32)
    A["col_idx"], A["val"] = A["col_idx"][:keep], A["val"][:keep]
    M, (row, col, val) = _coo_on_device(gko, A, dev)
    n, m, nnz = A["n_rows"], A["n_cols"], keep
    assert nnz % 4 != 0 and nnz > 3 * 2816
    for call, seed in enumerate((5, 6)):  # two calls in a row, different inputs
        x_h = syn.vector(m, seed)
        y0_h = syn.vector(n, seed + 10)
        x = torch.from_numpy(x_h).to(dev)
        y_ref = torch.from_numpy(y0_h).to(dev)
        M.spmv(x, y_ref, alpha, beta, fmt="coo")
        y = torch.from_numpy(y0_h).to(dev)
        err = torch.zeros(1, dtype=torch.int32, device=dev)
        gko.gko_spmv_coo_noalloc(n, m, nnz, row.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr(),
                                 y.data_ptr(), alpha, beta, err.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        ref, mag = orc.spmv_dot2(A, x_h, alpha, beta, y0_h)
        d = np.abs(y.cpu().numpy() - ref)
        assert np.all(d <= 1e-12 * mag + 1e-300), (call, float(d.max()))
        d_handle = np.abs(y_ref.cpu().numpy() - ref)
        assert np.all(d_handle <= 1e-12 * mag + 1e-300), (call, float(d_handle.max()))
        assert int(err.item()) == 0


def test_no_alloc_limits_and_arguments(gko, dev):
    import torch
    b = gko.binding
    cap = b.lib.gko_spmv_coo_noalloc
    big = 32768 * 2816 + 1
    # beyond the fixed scratch: refused before any device work
    assert cap(10, 10, big, 16, 16, 16, 16, 16, 1.0, 0.0, None, None) == b.ERR_INVALID_ARG
    assert "scratch" in b.last_error()
    # misaligned arrays are refused
    buf = torch.zeros(64, dtype=torch.int32, device=dev)
    v = torch.zeros(64, dtype=torch.float64, device=dev)
    assert cap(4, 4, 4, buf.data_ptr() + 4, buf.data_ptr(), v.data_ptr(), v.data_ptr(), v.data_ptr(), 1.0, 0.0,
               None, None) == b.ERR_INVALID_ARG
    # no entries: y = beta * y
    y = torch.full((5,), 2.0, dtype=torch.float64, device=dev)
    gko.gko_spmv_coo_noalloc(5, 5, 0, 0, 0, 0, 0, y.data_ptr(), 1.0, 0.5)
    torch.cuda.synchronize()
    assert torch.all(y == 1.0)


def test_no_alloc_at_the_entry_limit(gko, dev):
    """nnz exactly GKO_NOALLOC_MAX_TILES * 2816 is accepted and runs in the
    fixed array (its last tile, index 32767, carries a row into the fix-up).
    Rows of 3001 entries cross tile boundaries; values 1 and x_c = (c mod 7)
    - 3 make every row sum an exact integer: y_r = sum_{c < len_r} x_c."""
    import torch
    nnz = 32768 * 2816
    L, m = 3001, 4096
    n = (nnz + L - 1) // L
    k = torch.arange(nnz, device=dev, dtype=torch.int64)
    row = (k // L).to(torch.int32)
    col = (k % L).to(torch.int32)
    del k
    val = torch.ones(nnz, dtype=torch.float64, device=dev)
    xc = (np.arange(m) % 7 - 3).astype(np.float64)
    x = torch.from_numpy(xc).to(dev)
    y = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    gko.gko_spmv_coo_noalloc(n, m, nnz, row.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr(), y.data_ptr(),
                             1.0, 0.0, err.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    exp = np.full(n, xc[:L].sum())
    exp[-1] = xc[:nnz - (n - 1) * L].sum()
    assert np.array_equal(y.cpu().numpy(), exp)
    b = gko.binding
    assert b.lib.gko_spmv_coo_noalloc(n, m, nnz + 1, row.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr(),
                                      y.data_ptr(), 1.0, 0.0, None, None) == b.ERR_INVALID_ARG


def test_no_alloc_on_a_second_device(gko, dev, orc):
    """The array's address is looked up per device: a call on device 1 after
    calls on device 0 matches the oracle too."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("one device")
    A = syn.powerlaw(20000, 12.0, 1.5, 900, seed=93)
    n, m = A["n_rows"], A["n_cols"]
    rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(A["row_ptr"]))
    x_h = syn.vector(m, 2)
    ref, mag = orc.spmv_dot2(A, x_h)
    for d in (0, 1):
        with torch.cuda.device(d):
            dv = torch.device("cuda", d)
            r, c, v = (torch.from_numpy(np.ascontiguousarray(a)).to(dv) for a in (rows, A["col_idx"], A["val"]))
            x = torch.from_numpy(x_h).to(dv)
            y = torch.empty(n, dtype=torch.float64, device=dv)
            gko.gko_spmv_coo_noalloc(n, m, len(A["val"]), r.data_ptr(), c.data_ptr(), v.data_ptr(), x.data_ptr(),
                                     y.data_ptr(), 1.0, 0.0, None, torch.cuda.current_stream(dv).cuda_stream)
            torch.cuda.synchronize(dv)
            assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * mag + 1e-300)
