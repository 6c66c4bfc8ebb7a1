"""Failure detection without a GPU fault.

The staged kernels wait for each tile's bulk copy with a bounded poll loop.
gko_set_wait_limit(0) makes that first wait give up at once, so the timeout
path runs deterministically: the kernel sets bit 0 of the error word, waits
(with the normal limit) for its copies still in flight and exits; nothing
hangs and the context stays usable.  The bounds-checked build of the library
(GKO_CHECK_BOUNDS) reports an out-of-range index of the allocation-free COO
entry as bit 1 and skips the entry instead of reading out of range; the bad
index is planted on the host.
"""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

DEFAULT = 0xFFFFFFFF


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.fixture
def no_wait(gko):
    gko.binding.gko_set_wait_limit(0)
    yield
    gko.binding.gko_set_wait_limit(DEFAULT)


def test_timeout_marks_spmv_and_leaves_context_usable(gko, dev, orc):
    import torch
    A = syn.powerlaw(40000, 12.0, 1.5, 900, seed=5)
    n = A["n_rows"]
    M = gko.Matrix(A)
    M.convert("coo")
    x_h = syn.vector(n, 3)
    x = _t(x_h, dev)
    y = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    gko.binding.gko_set_wait_limit(0)
    try:
        M.spmv(x, y, fmt="coo")
        torch.cuda.synchronize()
    finally:
        gko.binding.gko_set_wait_limit(DEFAULT)
    assert M.errors(clear=True) & 1  # bit 0: a bounded wait gave up
    assert bool(torch.isnan(y).any())  # the output was not produced
    # the same handle and context work again at the default limit
    M.spmv(x, y, fmt="coo")
    torch.cuda.synchronize()
    ref, mag = orc.spmv_dot2(A, x_h)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * mag + 1e-300)
    assert M.errors() == 0


def test_timeout_stops_cg_with_status(gko, dev, orc, no_wait):
    # rows of 16 entries: the single-reduction CG runs its CSR product in the
    # staged row-block kernel; COO products go through the segmented kernel.
    # The first product gives up, so the matrix need not be SPD.
    A = syn.banded(20000, 64, 16, seed=3)
    n = A["n_rows"]
    b = _t(orc.spmv_csr(A, syn.vector(n, 4)), dev)
    for solve, fmt in (("cg_single_reduction", "csr"), ("cg", "coo")):
        M = gko.Matrix(A)
        if fmt != "csr":
            M.convert(fmt)
        x = _t(np.zeros(n), dev)
        with pytest.raises(gko.GkoError) as e:
            getattr(M, solve)(b, x, tol=1e-10, maxit=500, fmt=fmt)
        assert e.value.status == gko.binding.ERR_TIMEOUT, (solve, e.value)
        assert M.errors(clear=True) & 1


def test_timeout_stops_mixed_cg_with_status(gko, dev, orc, no_wait):
    # the inner product of mixed CG streams an ELL copy of A_lo by bulk copies
    A = syn.diffusion7(24, 1.0, seed=6)
    n = A["n_rows"]
    b = _t(orc.spmv_csr(A, syn.vector(n, 4)), dev)
    M = gko.Matrix(A)
    x = _t(np.zeros(n), dev)
    with pytest.raises(gko.GkoError) as e:
        M.cg_mixed(b, x, inner="fp32", tol=1e-10)
    assert e.value.status == gko.binding.ERR_TIMEOUT


def test_checked_build_reports_bad_column(gko, dev, orc):
    import ctypes as C

    import torch
    lib = gko.binding.checked_lib()
    A = syn.powerlaw(30000, 10.0, 1.5, 700, seed=12)
    n, m = A["n_rows"], A["n_cols"]
    rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(A["row_ptr"]))
    col = A["col_idx"].copy()
    val = A["val"].copy()
    bad = [7, len(col) // 2, len(col) - 2]
    col[bad[0]] = m + 5      # past the end
    col[bad[1]] = -3         # negative
    col[bad[2]] = 1 << 30    # far past the end
    nnz = len(val)
    x_h = syn.vector(m, 8)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    r_d, c_d, v_d, x_d = _t(rows, dev), _t(col, dev), _t(val, dev), _t(x_h, dev)
    st = lib.gko_spmv_coo_noalloc(n, m, nnz, r_d.data_ptr(), c_d.data_ptr(), v_d.data_ptr(), x_d.data_ptr(),
                                  y.data_ptr(), 1.0, 0.0, err.data_ptr(), C.c_void_p(0))
    assert st == gko.binding.OK
    torch.cuda.synchronize()
    assert int(err.item()) & 2  # bit 1: index out of range
    # the bad entries are skipped: the oracle's product with their values zeroed
    B = dict(A)
    B["val"] = val.copy()
    B["val"][bad] = 0.0
    ref, mag = orc.spmv_dot2(B, x_h)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * mag + 1e-300)
    # valid indices: no bit, same result as the unchecked library
    err.zero_()
    c_ok = _t(A["col_idx"], dev)
    st = lib.gko_spmv_coo_noalloc(n, m, nnz, r_d.data_ptr(), c_ok.data_ptr(), v_d.data_ptr(), x_d.data_ptr(),
                                  y.data_ptr(), 1.0, 0.0, err.data_ptr(), C.c_void_p(0))
    assert st == gko.binding.OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref, mag = orc.spmv_dot2(A, x_h)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * mag + 1e-300)
