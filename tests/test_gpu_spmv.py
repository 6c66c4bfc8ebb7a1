"""Parity of every SpMV kernel with the oracle (through the C ABI).

Tolerance (the spec bar, read per entry against the magnitude of the
terms): |y_gpu - y_ref| <= 1e-12 * (|alpha| |A| |x| + |beta| |y|)_i, with
y_ref the oracle's compensated (Dot2) result.  Integer-valued inputs make
every partial sum exact, so there all kernels must agree bit for bit."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

FORMATS = ("csr", "coo", "ell", "sellp", "hybrid")
CSR_CONFIGS = (1, 2, 3, 4, 5, 6, 7, 10)  # subwarp 1..32, load-balanced, binned


def mats():
    return {
        "tiny": syn.random_csr(1, 1, 1, seed=1),
        "ragged": syn.random_csr(1001, 997, 40, seed=2, empty_frac=0.3),
        "wide": syn.random_csr(300, 5000, 200, seed=3),
        "empty_rows_many": syn.random_csr(20000, 20000, 3, seed=4, empty_frac=0.9),
        "powerlaw": syn.powerlaw(30000, 20.0, 1.5, 5000, seed=5),
        "long_row": _long_row(),
        "stencil": syn.stencil27(20, seed=6),
        "banded": syn.banded(20000, 64, 16, seed=7),
        "blockdiag": syn.block_diagonal(8000, 8, seed=8),
        "all_empty": syn.random_csr(100, 100, 0, seed=9),
    }


def _long_row():
    """One row of 20000 entries among short rows: spans several tiles."""
    A = syn.random_csr(5000, 30000, 4, seed=10)
    rp = A["row_ptr"].astype(np.int64)
    L = np.diff(rp)
    L[2500] = 20000
    cols = []
    for i in range(5000):
        if i == 2500:
            cols.append(np.arange(0, 30000, 1.5).astype(np.int64)[:20000])
        else:
            cols.append(A["col_idx"][rp[i]:rp[i + 1]])
    col = np.concatenate(cols).astype(np.int32)
    row_ptr = np.concatenate([[0], np.cumsum(L)]).astype(np.int32)
    return dict(n_rows=5000, n_cols=30000, row_ptr=row_ptr, col_idx=col,
                val=syn.uniform_pm1(10, syn.S_VAL, np.arange(len(col), dtype=np.uint64)))


@pytest.fixture(scope="module")
def handles(gko, dev):
    out = {}
    for name, A in mats().items():
        M = gko.Matrix(A)
        for f in ("coo", "hybrid"):
            M.convert(f)
        for f in ("ell", "sellp"):  # padded formats may be refused
            try:
                M.convert(f)
            except gko.GkoError as e:
                assert e.status == gko.binding.ERR_FORMAT_TOO_LARGE
        out[name] = (A, M)
    return out


def _run(M, f, x, y0, alpha, beta, dev, config=0):
    import torch
    xd = torch.from_numpy(x).to(dev)
    yd = torch.from_numpy(y0.copy()).to(dev)
    M.spmv(xd, yd, alpha, beta, fmt=f, config=config)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0), (2.5, -0.5), (0.0, 1.5)])
def test_formats_match_oracle(gko, dev, handles, orc, alpha, beta):
    for name, (A, M) in handles.items():
        x = syn.vector(A["n_cols"], 11)
        y0 = syn.vector(A["n_rows"], 12)
        ref, mag = orc.spmv_dot2(A, x, alpha, beta, y0)
        for f in FORMATS:
            if not M.has(f):
                continue
            y = _run(M, f, x, y0, alpha, beta, dev)
            err = np.abs(y - ref)
            bad = np.nonzero(~(err <= 1e-12 * mag + 1e-300))[0]
            assert bad.size == 0, (name, f, bad[:5], err[bad[:5]], mag[bad[:5]])
        assert M.errors() == 0


def _applies(A, cfg):
    """Row-block kernels need max row length <= 128; banded also max |i-j| <= 1024."""
    L = np.diff(A["row_ptr"])
    if L.sum() == 0:  # no stored entry: every configuration reduces to y = beta y
        return True
    if cfg in (8, 9) and not (1 <= L.max(initial=0) <= 128):
        return False
    if cfg == 8:
        rows = np.repeat(np.arange(A["n_rows"]), L)
        return np.abs(A["col_idx"].astype(np.int64) - rows).max(initial=0) <= 1024
    return True


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 2.0)])
def test_csr_configs_match_oracle(gko, dev, handles, orc, alpha, beta):
    for name, (A, M) in handles.items():
        x = syn.vector(A["n_cols"], 13)
        y0 = syn.vector(A["n_rows"], 14)
        ref, mag = orc.spmv_dot2(A, x, alpha, beta, y0)
        for cfg in CSR_CONFIGS + (8, 9):
            if not _applies(A, cfg):
                with pytest.raises(gko.GkoError):
                    _run(M, "csr", x, y0, alpha, beta, dev, config=cfg)
                continue
            y = _run(M, "csr", x, y0, alpha, beta, dev, config=cfg)
            assert np.all(np.abs(y - ref) <= 1e-12 * mag + 1e-300), (name, cfg)


def test_banded_kernel_with_unaligned_x(gko, dev, orc):
    """x at an 8-byte (not 16-byte) offset: the banded kernel must fall back
    to gathers through L1/L2 and still be exact."""
    import torch
    A = syn.banded(5000, 64, 16, seed=77)
    M = gko.Matrix(A)
    x = syn.vector(A["n_cols"], 78)
    xbuf = torch.zeros(A["n_cols"] + 1, dtype=torch.float64, device=dev)
    xbuf[1:] = torch.from_numpy(x).to(dev)
    xv = xbuf[1:]
    assert xv.data_ptr() % 16 == 8
    y = torch.zeros(A["n_rows"], dtype=torch.float64, device=dev)
    M.spmv(xv, y, config=8)
    ref, mag = orc.spmv_dot2(A, x)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * mag)


def test_beta_zero_overwrites_nan(gko, dev, handles):
    for name, (A, M) in handles.items():
        x = syn.vector(A["n_cols"], 15)
        y0 = np.full(A["n_rows"], np.nan)
        for f in FORMATS:
            if M.has(f):
                y = _run(M, f, x, y0, 1.0, 0.0, dev)
                assert np.all(np.isfinite(y)), (name, f)


def test_integer_inputs_bit_exact_across_kernels(gko, dev, orc):
    A = syn.powerlaw(20000, 20.0, 1.5, 3000, seed=21)
    A["val"] = np.round(A["val"] * 16.0)
    x = np.round(syn.vector(A["n_cols"], 22) * 64.0)
    exact = orc.spmv_csr(A, x)  # every partial sum is an integer below 2^53
    M = gko.Matrix(A)
    M.set_params(ell_factor=1000.0)  # allow the padded formats on this skewed matrix
    for f in ("coo", "sellp", "hybrid", "ell"):
        M.convert(f)
    y0 = np.zeros(A["n_rows"])
    for f in ("csr", "coo", "sellp", "hybrid", "ell"):
        assert np.array_equal(_run(M, f, x, y0, 1.0, 0.0, dev), exact), f
    for cfg in CSR_CONFIGS:
        assert np.array_equal(_run(M, "csr", x, y0, 1.0, 0.0, dev, config=cfg), exact), cfg


def test_ell_refused_when_padding_is_too_large(gko, dev):
    A = syn.powerlaw(200000, 20.0, 1.5, 20000, seed=4)
    M = gko.Matrix(A)
    with pytest.raises(gko.GkoError) as e:
        M.convert("ell")
    assert e.value.status == gko.binding.ERR_FORMAT_TOO_LARGE
    import torch
    x = torch.zeros(A["n_cols"], dtype=torch.float64, device=dev)
    y = torch.zeros(A["n_rows"], dtype=torch.float64, device=dev)
    with pytest.raises(gko.GkoError) as e:
        M.spmv(x, y, fmt="ell")
    assert e.value.status == gko.binding.ERR_FORMAT_UNAVAILABLE


def test_invalid_csr_is_rejected(gko, dev):
    A = syn.random_csr(50, 50, 5, seed=30)
    bad = dict(A)
    bad["col_idx"] = A["col_idx"].copy()
    bad["col_idx"][3] = 50  # out of range
    with pytest.raises(gko.GkoError) as e:
        gko.Matrix(bad)
    assert e.value.status == gko.binding.ERR_INVALID_MATRIX
    bad = dict(A)
    bad["row_ptr"] = A["row_ptr"].copy()
    bad["row_ptr"][10], bad["row_ptr"][11] = bad["row_ptr"][11] + 1, bad["row_ptr"][10]
    with pytest.raises(gko.GkoError):
        gko.Matrix(bad)


def test_host_entry_point_matches_device(gko, dev, orc):
    A = syn.banded(10000, 64, 16, seed=31)
    M = gko.Matrix(A)
    x = syn.vector(A["n_cols"], 32)
    y0 = syn.vector(A["n_rows"], 33)
    ref, mag = orc.spmv_dot2(A, x, 2.0, 0.5, y0)
    y = y0.copy()
    M.spmv_host(x, y, 2.0, 0.5)
    assert np.all(np.abs(y - ref) <= 1e-12 * mag)


@pytest.mark.parametrize("name", ["stencil27_128", "banded_4M", "powerlaw_2M", "blockdiag_1M"])
def test_full_size_sampled_rows(gko, dev, orc, name):
    """The benchmark matrices at full size, in the launch configuration the
    benchmark times (alpha = 1, beta = 0): 2000 sampled rows per format
    against the oracle's compensated sum of the same rows."""
    import torch
    A = syn.workload(name)
    M = gko.Matrix(A)
    for f in ("coo", "sellp", "hybrid", "ell"):
        try:
            M.convert(f)
        except gko.GkoError as e:
            assert f in ("ell", "sellp") and e.status == gko.binding.ERR_FORMAT_TOO_LARGE
    x = syn.vector(A["n_cols"], 99)
    rows = np.unique(np.concatenate([np.linspace(0, A["n_rows"] - 1, 1500).astype(np.int64),
                                     np.argsort(np.diff(A["row_ptr"]))[-500:]]))
    rp = A["row_ptr"].astype(np.int64)
    sub_rp = np.concatenate([[0], np.cumsum(rp[rows + 1] - rp[rows])]).astype(np.int32)
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    S = dict(n_rows=len(rows), n_cols=A["n_cols"], row_ptr=sub_rp, col_idx=A["col_idx"][idx], val=A["val"][idx])
    ref, mag = orc.spmv_dot2(S, x)
    xd = torch.from_numpy(x).to(dev)
    yd = torch.empty(A["n_rows"], dtype=torch.float64, device=dev)
    for f in ("csr", "coo", "ell", "sellp", "hybrid"):
        if not M.has(f):
            continue
        yd.fill_(float("nan"))
        M.spmv(xd, yd, fmt=f)
        y = yd.cpu().numpy()
        assert np.all(np.isfinite(y)), f
        assert np.all(np.abs(y[rows] - ref) <= 1e-12 * mag), f
    assert M.errors() == 0
