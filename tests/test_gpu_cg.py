"""CG on the GPU against the oracle.  Iterates differ by rounding, so
parity means: both reach the true relative residual, iteration counts agree
within max(5, 2 %), and the GPU solution's error against the manufactured
solution is within 10x of the oracle's own."""
import math

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("fmt", ["csr", "coo", "ell", "sellp", "hybrid"])
def test_cg_laplace_128(gko, dev, orc, fmt):
    A = syn.laplace2d(128)
    n = A["n_rows"]
    xt = syn.vector(n, 1)
    b = orc.spmv_csr(A, xt)
    x_o, st_o, it_o, res_o = orc.cg(A, b, tol=1e-10)
    M = gko.Matrix(A)
    if fmt != "csr":
        M.convert(fmt)
    x = _t(np.zeros(n), dev)
    info = M.cg(_t(b, dev), x, tol=1e-10, maxit=10000, fmt=fmt)
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert abs(info.iterations - it_o) <= max(5, 0.02 * it_o), (info.iterations, it_o)
    xg = x.cpu().numpy()
    assert orc.true_rel_residual(A, b, xg) <= 1e-10
    e_o = np.linalg.norm(x_o - xt) / np.linalg.norm(xt)
    e_g = np.linalg.norm(xg - xt) / np.linalg.norm(xt)
    assert e_g <= 10 * e_o + 1e-15


@pytest.mark.parametrize("fmt", ["csr", "ell"])
def test_cg_unaligned_solution_vector(gko, dev, orc, fmt):
    """x 8 bytes off a 16-byte boundary takes the scalar update kernels; the
    same solve from an aligned x takes the 128-bit ones: both match the
    oracle (odd n, so the vector loops also leave a tail)."""
    import torch
    A = syn.diffusion7(17, 1.0, seed=6)
    n = A["n_rows"]
    assert n % 2 == 1
    xt = syn.vector(n, 3)
    b = orc.spmv_csr(A, xt)
    x_o, _, it_o, _ = orc.cg(A, b, tol=1e-10)
    M = gko.Matrix(A)
    if fmt != "csr":
        M.convert(fmt)
    buf = torch.zeros(n + 1, dtype=torch.float64, device=dev)
    for x in (buf[:n], buf[1:]):
        x.zero_()
        info = M.cg(_t(b, dev), x, tol=1e-10, fmt=fmt)
        assert info.status == 0 and abs(info.iterations - it_o) <= max(5, 0.02 * it_o)
        xg = x.cpu().numpy()
        assert orc.true_rel_residual(A, b, xg) <= 1e-10
        assert np.linalg.norm(xg - x_o) <= 1e-8 * np.linalg.norm(x_o)


def _skewed_spd(n, seed):
    """SPD matrix with power-law row lengths: the symmetrised pattern of a
    power-law matrix, off-diagonals -|a|, diagonal 1 + sum of |off-diagonals|
    (strictly diagonally dominant)."""
    sp = pytest.importorskip("scipy.sparse")
    P = syn.powerlaw(n, 6.0, 1.5, n // 4, seed=seed)
    M = sp.csr_matrix((np.abs(P["val"]), P["col_idx"], P["row_ptr"]), shape=(n, n))
    M = (M + M.T).tolil()
    M.setdiag(0.0)
    M = -M.tocsr()
    M.eliminate_zeros()
    d = 1.0 + np.asarray(abs(M).sum(axis=1)).ravel()
    M = (M + sp.diags(d)).tocsr()
    M.sort_indices()
    return dict(n_rows=n, n_cols=n, row_ptr=M.indptr.astype(np.int32), col_idx=M.indices.astype(np.int32),
                val=M.data.astype(np.float64))


@pytest.mark.parametrize("fmt", ["csr", "coo", "ell", "sellp", "hybrid"])
def test_cg_single_reduction_laplace_128(gko, dev, orc, fmt):
    A = syn.laplace2d(128)
    n = A["n_rows"]
    xt = syn.vector(n, 1)
    b = orc.spmv_csr(A, xt)
    x_o, st_o, it_o, res_o = orc.cg_single_reduction(A, b, tol=1e-10)
    _, _, it_hs, _ = orc.cg(A, b, tol=1e-10)
    M = gko.Matrix(A)
    if fmt != "csr":
        M.convert(fmt)
    x = _t(np.zeros(n), dev)
    info = M.cg_single_reduction(_t(b, dev), x, tol=1e-10, maxit=10000, fmt=fmt)
    assert info.status == 0 and info.rel_residual <= 1e-10
    for it in (it_o, it_hs):
        assert abs(info.iterations - it) <= max(5, 0.02 * it), (info.iterations, it)
    xg = x.cpu().numpy()
    assert orc.true_rel_residual(A, b, xg) <= 1e-10
    e_o = np.linalg.norm(x_o - xt) / np.linalg.norm(xt)
    e_g = np.linalg.norm(xg - xt) / np.linalg.norm(xt)
    assert e_g <= 10 * e_o + 1e-15


def test_cg_single_reduction_skewed_rows(gko, dev, orc):
    """Rows of very different lengths: the product is the load-balanced
    kernel plus a separate dot launch (not the fused row-block kernel)."""
    A = _skewed_spd(20000, 31)
    n = A["n_rows"]
    lens = np.diff(A["row_ptr"])
    assert lens.max() > 2 * lens.mean() + 16  # the row-block kernel does not apply
    xt = syn.vector(n, 5)
    b = orc.spmv_csr(A, xt)
    x_o, st_o, it_o, res_o = orc.cg_single_reduction(A, b, tol=1e-10)
    assert st_o == 0
    M = gko.Matrix(A)
    for solve in (M.cg, M.cg_single_reduction):
        x = _t(np.zeros(n), dev)
        info = solve(_t(b, dev), x, tol=1e-10, maxit=5000)
        assert info.status == 0 and info.rel_residual <= 1e-10
        assert abs(info.iterations - it_o) <= max(5, 0.02 * it_o), (info.iterations, it_o)
        assert orc.true_rel_residual(A, b, x.cpu().numpy()) <= 1e-10


def test_cg_single_reduction_special_cases(gko, dev, orc):
    A = syn.laplace2d(16)
    n = A["n_rows"]
    M = gko.Matrix(A)
    x = _t(np.ones(n), dev)
    info = M.cg_single_reduction(_t(np.zeros(n), dev), x)
    assert info.status == 0 and info.iterations == 0 and float(x.abs().max()) == 0.0
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x = _t(np.zeros(n), dev)
    info = M.cg_single_reduction(_t(b, dev), x, maxit=3)
    assert info.status == gko.binding.ERR_NOT_CONVERGED and info.iterations == 3
    xo, _, _, _ = orc.cg_single_reduction(A, b, maxit=3)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-12 * np.linalg.norm(xo)
    x = _t(syn.vector(n, 2), dev)
    info = M.cg_single_reduction(_t(b, dev), x)
    assert info.status == 0 and info.iterations == 0
    N = dict(A)
    N["val"] = -A["val"]
    x = _t(np.zeros(n), dev)
    info = gko.Matrix(N).cg_single_reduction(_t(b, dev), x)
    assert info.status == gko.binding.ERR_BREAKDOWN
    bn = b.copy()
    bn[5] = np.nan
    x = _t(np.zeros(n), dev)
    info = M.cg_single_reduction(_t(bn, dev), x)
    assert info.status == gko.binding.ERR_BREAKDOWN


@pytest.mark.parametrize("fmt", ["csr", "ell", "hybrid"])
def test_pcg_jacobi_scaled_operator(gko, dev, orc, fmt):
    """Diffusion operator rescaled by a diagonal spanning three decades: the
    GPU's Jacobi PCG matches the oracle's step count and both reach the
    manufactured solution; plain CG needs several times more steps."""
    A0 = syn.diffusion7(24, 1.0, seed=6)
    n = A0["n_rows"]
    s = 10.0 ** (3.0 * syn.uniform01(25, 1, np.arange(n, dtype=np.uint64)))
    rows = np.repeat(np.arange(n), np.diff(A0["row_ptr"]))
    A = dict(A0)
    A["val"] = A0["val"] * s[rows] * s[A0["col_idx"]]
    xt = syn.vector(n, 26)
    b = orc.spmv_csr(A, xt)
    x_o, st_o, it_o, res_o = orc.pcg_jacobi(A, b, tol=1e-10, maxit=20000)
    assert st_o == 0
    M = gko.Matrix(A)
    if fmt != "csr":
        M.convert(fmt)
    x = _t(np.zeros(n), dev)
    info = M.pcg_jacobi(_t(b, dev), x, tol=1e-10, maxit=20000, fmt=fmt)
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert abs(info.iterations - it_o) <= max(5, 0.02 * it_o), (info.iterations, it_o)
    xg = x.cpu().numpy()
    assert orc.true_rel_residual(A, b, xg) <= 1e-10
    e_o = np.linalg.norm(x_o - xt) / np.linalg.norm(xt)
    assert np.linalg.norm(xg - xt) / np.linalg.norm(xt) <= 10 * e_o + 1e-15
    x2 = _t(np.zeros(n), dev)
    info_cg = M.cg(_t(b, dev), x2, tol=1e-10, maxit=2000, fmt=fmt)
    assert info_cg.iterations > 3 * info.iterations


def test_pcg_jacobi_special_cases(gko, dev, orc):
    A = syn.laplace2d(16)
    n = A["n_rows"]
    M = gko.Matrix(A)
    x = _t(np.ones(n), dev)
    info = M.pcg_jacobi(_t(np.zeros(n), dev), x)
    assert info.status == 0 and info.iterations == 0 and float(x.abs().max()) == 0.0
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x = _t(np.zeros(n), dev)
    info = M.pcg_jacobi(_t(b, dev), x, maxit=3)
    assert info.status == gko.binding.ERR_NOT_CONVERGED and info.iterations == 3
    xo, _, _, _ = orc.pcg_jacobi(A, b, maxit=3)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-12 * np.linalg.norm(xo)
    # constant diagonal: the same steps as plain CG
    x = _t(np.zeros(n), dev)
    info = M.pcg_jacobi(_t(b, dev), x, tol=1e-10)
    x2 = _t(np.zeros(n), dev)
    info2 = M.cg(_t(b, dev), x2, tol=1e-10)
    assert abs(info.iterations - info2.iterations) <= 1
    # a zero diagonal entry: breakdown before any step
    Z = dict(A)
    rows = np.repeat(np.arange(n), np.diff(A["row_ptr"]))
    Z["val"] = np.where((A["col_idx"] == rows) & (rows == 7), 0.0, A["val"])
    x = _t(np.zeros(n), dev)
    info = gko.Matrix(Z).pcg_jacobi(_t(b, dev), x)
    assert info.status == gko.binding.ERR_BREAKDOWN and info.iterations == 0


def test_cg_special_cases(gko, dev, orc):
    A = syn.laplace2d(16)
    n = A["n_rows"]
    M = gko.Matrix(A)
    # b = 0 -> x = 0 at once
    x = _t(np.ones(n), dev)
    info = M.cg(_t(np.zeros(n), dev), x)
    assert info.status == 0 and info.iterations == 0 and float(x.abs().max()) == 0.0
    # maxit reached
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x = _t(np.zeros(n), dev)
    info = M.cg(_t(b, dev), x, maxit=3)
    assert info.status == gko.binding.ERR_NOT_CONVERGED and info.iterations == 3
    # exact initial guess: no iteration
    x = _t(syn.vector(n, 2), dev)
    info = M.cg(_t(b, dev), x)
    assert info.status == 0 and info.iterations == 0
    # not SPD -> breakdown reported, no hang
    N = dict(A)
    N["val"] = -A["val"]
    MN = gko.Matrix(N)
    x = _t(np.zeros(n), dev)
    info = MN.cg(_t(b, dev), x)
    assert info.status == gko.binding.ERR_BREAKDOWN
    # NaN in b -> breakdown, no hang
    bn = b.copy()
    bn[5] = np.nan
    x = _t(np.zeros(n), dev)
    info = M.cg(_t(bn, dev), x)
    assert info.status == gko.binding.ERR_BREAKDOWN


def test_cg_small_spd_vs_cholesky(gko, dev, orc):
    B = syn.batched_spd(5, seed=50, n_min=20, n_max=200)
    for s in range(5):
        r0, r1 = B["row_off"][s], B["row_off"][s + 1]
        k0, k1 = B["row_ptr"][r0], B["row_ptr"][r1]
        A = dict(n_rows=r1 - r0, n_cols=r1 - r0, row_ptr=(B["row_ptr"][r0:r1 + 1] - k0).astype(np.int32),
                 col_idx=B["col_idx"][k0:k1], val=B["val"][k0:k1])
        D = orc.to_dense(A)
        b = B["rhs"][r0:r1]
        xc, st = orc.cholesky_solve(D, b)
        M = gko.Matrix(A)
        x = _t(np.zeros(r1 - r0), dev)
        info = M.cg(_t(b, dev), x, tol=1e-12)
        assert info.status == 0
        assert np.linalg.norm(x.cpu().numpy() - xc) <= 1e-10 * np.linalg.norm(xc)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_cg_matches_oracle(gko, dev, orc, prec):
    A = syn.diffusion7(40, 1.0, seed=6)
    n = A["n_rows"]
    xt = syn.vector(n, 6)
    b = orc.spmv_csr(A, xt)
    x64, st, it64, res64 = orc.cg(A, b, tol=1e-10)
    xo, st_o, outer_o, inner_o, res_o = orc.cg_mixed(A, b, prec, tol=1e-10, inner_tol=1e-3)
    assert st_o == 0
    M = gko.Matrix(A)
    x = _t(np.zeros(n), dev)
    info = M.cg_mixed(_t(b, dev), x, inner=prec, tol=1e-10, inner_tol=1e-3)
    assert info.status == 0 and info.rel_residual <= 1e-10
    xg = x.cpu().numpy()
    assert orc.true_rel_residual(A, b, xg) <= 1e-10
    assert abs(info.outer_iterations - outer_o) <= 2, (info.outer_iterations, outer_o)
    e_ref = np.linalg.norm(x64 - xt)
    assert np.linalg.norm(xg - xt) <= 10 * e_ref + 1e-14 * np.linalg.norm(xt)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_cg_skewed_rows(gko, dev, orc, prec):
    """Inner product by the load-balanced kernel + separate dots."""
    A = _skewed_spd(20000, 32)
    n = A["n_rows"]
    xt = syn.vector(n, 7)
    b = orc.spmv_csr(A, xt)
    xo, st_o, outer_o, inner_o, res_o = orc.cg_mixed(A, b, prec, tol=1e-10, inner_tol=1e-3)
    assert st_o == 0
    M = gko.Matrix(A)
    x = _t(np.zeros(n), dev)
    info = M.cg_mixed(_t(b, dev), x, inner=prec, tol=1e-10, inner_tol=1e-3)
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert orc.true_rel_residual(A, b, x.cpu().numpy()) <= 1e-10
    assert abs(info.outer_iterations - outer_o) <= 2, (info.outer_iterations, outer_o)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_cg_wide_band(gko, dev, orc, prec):
    """Symmetrically permuted diffusion operator: short uniform rows but
    |i - j| up to n > 32767, so the inner ELL copy keeps int32 columns."""
    sp = pytest.importorskip("scipy.sparse")
    A0 = syn.diffusion7(34, 1.0, seed=9)
    n = A0["n_rows"]
    perm = np.random.default_rng(5).permutation(n)
    M0 = sp.csr_matrix((A0["val"], A0["col_idx"], A0["row_ptr"]), shape=(n, n))
    Mp = M0[perm][:, perm].tocsr()
    Mp.sort_indices()
    A = dict(n_rows=n, n_cols=n, row_ptr=Mp.indptr.astype(np.int32), col_idx=Mp.indices.astype(np.int32),
             val=Mp.data.astype(np.float64))
    assert np.max(np.abs(A["col_idx"] - np.repeat(np.arange(n), np.diff(A["row_ptr"])))) > 32767
    xt = syn.vector(n, 8)
    b = orc.spmv_csr(A, xt)
    xo, st_o, outer_o, inner_o, res_o = orc.cg_mixed(A, b, prec, tol=1e-10, inner_tol=1e-3)
    assert st_o == 0
    M = gko.Matrix(A)
    x = _t(np.zeros(n), dev)
    info = M.cg_mixed(_t(b, dev), x, inner=prec, tol=1e-10, inner_tol=1e-3)
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert orc.true_rel_residual(A, b, x.cpu().numpy()) <= 1e-10
    assert abs(info.outer_iterations - outer_o) <= 2, (info.outer_iterations, outer_o)


@pytest.mark.parametrize("prec,case", [("fp32", "scaled"), ("bf16", "diffusion"), ("fp32", "skewed")])
def test_mixed_cg_jacobi(gko, dev, orc, prec, case):
    """Jacobi-preconditioned inner solve against the oracle's: outer
    corrections within 2, both at the FP64 residual; paths: ELL inner copy
    (scaled / variable-coefficient diffusion) and load-balanced product +
    dot kernel (skewed rows)."""
    if case == "skewed":
        A = _skewed_spd(20000, 33)
    else:
        A = syn.diffusion7(32, 1.0, seed=6)
        if case == "scaled":
            n = A["n_rows"]
            s = 10.0 ** (3.0 * syn.uniform01(27, 1, np.arange(n, dtype=np.uint64)))
            rows = np.repeat(np.arange(n), np.diff(A["row_ptr"]))
            A = dict(A)
            A["val"] = A["val"] * s[rows] * s[A["col_idx"]]
    n = A["n_rows"]
    xt = syn.vector(n, 30)
    b = orc.spmv_csr(A, xt)
    xo, st_o, outer_o, inner_o, res_o = orc.cg_mixed(A, b, prec, tol=1e-10, inner_tol=1e-2, precond="jacobi")
    assert st_o == 0
    M = gko.Matrix(A)
    x = _t(np.zeros(n), dev)
    info = M.cg_mixed(_t(b, dev), x, inner=prec, tol=1e-10, inner_tol=1e-2, precond="jacobi")
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert orc.true_rel_residual(A, b, x.cpu().numpy()) <= 1e-10
    assert abs(info.outer_iterations - outer_o) <= 2, (info.outer_iterations, outer_o)
    assert info.iterations <= 1.5 * inner_o + 20, (info.iterations, inner_o)


def test_lowprec_copy_matches_oracle_rounding(gko, dev, orc):
    """The mixed solver's rounded matrix is observable through its result on
    a system where one inner solve is exact: A_lo = A when every value is
    representable.  Here: check the rounding routines agree on the values
    of a diffusion operator by solving with inner_tol tiny and comparing
    the first correction is the same within FP32 noise."""
    A = syn.laplace2d(24)  # all values exact in BF16: A_lo == A
    n = A["n_rows"]
    b = orc.spmv_csr(A, syn.vector(n, 9))
    M = gko.Matrix(A)
    x = _t(np.zeros(n), dev)
    info = M.cg_mixed(_t(b, dev), x, inner="bf16", tol=1e-10, inner_tol=1e-6)
    assert info.status == 0 and info.outer_iterations <= 3


def test_batched_cg_matches_oracle(gko, dev, orc):
    import torch
    B = syn.batched_spd(300, seed=7)
    rhs = B["rhs"]
    xo, st_o, it_o, res_o = orc.cg_batched(B, rhs, tol=1e-10)
    assert np.all(st_o == 0)
    G = gko.Batch(B)
    # shared-memory layout (64..1024), register-resident layout (-128..-1024)
    # and the split layouts (p, or p and A p, in shared memory)
    P, PQ = gko.binding.BATCH_SHARED_P, gko.binding.BATCH_SHARED_PQ
    split = tuple(f | b for f in (P, PQ) for b in (32, 64, 128, 256))
    for bs in (0, 64, 128, 256, 512, 1024, -128, -256, -512, -1024) + split:
        x = torch.zeros(len(rhs), dtype=torch.float64, device=dev)
        s, infos = G.cg(_t(rhs, dev), x, tol=1e-10, maxit=1000, block_size=bs)
        assert s == 0, bs
        res = np.array([i.rel_residual for i in infos])
        its = np.array([i.iterations for i in infos])
        assert np.all(res <= 1e-10), bs
        assert np.all(np.abs(its - it_o) <= np.maximum(5, 0.02 * it_o)), bs
        xg = x.cpu().numpy()
        for s_ in range(0, 300, 37):
            r0, r1 = B["row_off"][s_], B["row_off"][s_ + 1]
            assert np.linalg.norm(xg[r0:r1] - xo[r0:r1]) <= 1e-8 * np.linalg.norm(xo[r0:r1])


def test_batched_cg_dense_cholesky_subset(gko, dev, orc):
    import torch
    B = syn.batched_spd(64, seed=70, n_min=32, n_max=300)
    G = gko.Batch(B)
    x = torch.zeros(len(B["rhs"]), dtype=torch.float64, device=dev)
    s, infos = G.cg(_t(B["rhs"], dev), x, tol=1e-12, maxit=1000)
    assert s == 0
    xg = x.cpu().numpy()
    for k in range(64):
        r0, r1 = B["row_off"][k], B["row_off"][k + 1]
        k0, k1 = B["row_ptr"][r0], B["row_ptr"][r1]
        A = dict(n_rows=r1 - r0, n_cols=r1 - r0, row_ptr=(B["row_ptr"][r0:r1 + 1] - k0).astype(np.int32),
                 col_idx=B["col_idx"][k0:k1], val=B["val"][k0:k1])
        xc, st = orc.cholesky_solve(orc.to_dense(A), B["rhs"][r0:r1])
        assert np.linalg.norm(xg[r0:r1] - xc) <= 1e-10 * np.linalg.norm(xc)


def _concat_batch(systems, rhs_seed):
    """One batch (the batched_spd layout) from a list of square CSR systems."""
    ro, rps, cis, vs, base = [0], [], [], [], 0
    for A in systems:
        rps.append(np.asarray(A["row_ptr"][:-1], np.int64) + base)
        cis.append(np.asarray(A["col_idx"], np.int32))
        vs.append(np.asarray(A["val"], np.float64))
        base += int(A["row_ptr"][-1])
        ro.append(ro[-1] + A["n_rows"])
    rp = np.concatenate(rps + [np.array([base], np.int64)]).astype(np.int32)
    ro = np.array(ro, np.int64)
    return dict(row_off=ro, row_ptr=rp, col_idx=np.concatenate(cis), val=np.concatenate(vs),
                sizes=np.diff(ro), rhs=syn.vector(int(ro[-1]), rhs_seed))


def _tiny(rows):
    rows = np.asarray(rows, np.float64)
    n = rows.shape[0]
    nz = [(i, j) for i in range(n) for j in range(n) if rows[i, j] != 0.0]
    rp = np.zeros(n + 1, np.int32)
    for i, _ in nz:
        rp[i + 1] += 1
    return dict(n_rows=n, n_cols=n, row_ptr=np.cumsum(rp).astype(np.int32),
                col_idx=np.array([j for _, j in nz], np.int32), val=np.array([rows[i, j] for i, j in nz]))


def test_batched_extreme_sizes_every_layout(gko, dev, orc):
    """Systems of 4,096 rows (the largest a batch takes), 2,025, 49, 2 and 1
    rows, and one with b = 0, in every layout that accepts them, against the
    oracle; the register layouts refuse systems above 1,024 rows."""
    import torch
    systems = [syn.laplace2d(64), _tiny([[2.0]]), _tiny([[2.0, -1.0], [-1.0, 2.0]]), syn.laplace2d(7),
               _tiny([[3.0, 1.0], [1.0, 3.0]]), syn.laplace2d(45)]
    B = _concat_batch(systems, 91)
    zero = 4  # system with a zero right-hand side
    r0z, r1z = B["row_off"][zero], B["row_off"][zero + 1]
    B["rhs"][r0z:r1z] = 0.0
    xo, st_o, it_o, _ = orc.cg_batched(B, B["rhs"], tol=1e-10, maxit=2000)
    assert np.all(st_o == 0) and B["row_off"][1] == 4096
    G = gko.Batch(B)
    x = torch.zeros(len(B["rhs"]), dtype=torch.float64, device=dev)
    with pytest.raises(gko.GkoError) as e:
        G.cg(_t(B["rhs"], dev), x, tol=1e-10, maxit=2000, block_size=-128)
    assert e.value.status == gko.binding.ERR_INVALID_ARG
    P, PQ = gko.binding.BATCH_SHARED_P, gko.binding.BATCH_SHARED_PQ
    for bs in (64, 128, 256, 512, 1024) + tuple(f | b for f in (P, PQ) for b in (32, 64, 128, 256)):
        x = torch.zeros(len(B["rhs"]), dtype=torch.float64, device=dev)
        x[r0z:r1z] = 0.5  # b = 0 returns x = 0 whatever the initial guess
        s, infos = G.cg(_t(B["rhs"], dev), x, tol=1e-10, maxit=2000, block_size=bs)
        assert s == 0, gko.binding.batch_layout(bs)
        xg = x.cpu().numpy()
        for k in range(len(systems)):
            r0, r1 = B["row_off"][k], B["row_off"][k + 1]
            if k == zero:
                assert infos[k].iterations == 0 and infos[k].rel_residual == 0.0 and np.all(xg[r0:r1] == 0.0)
                continue
            assert infos[k].rel_residual <= 1e-10, (bs, k)
            assert abs(infos[k].iterations - it_o[k]) <= max(5, 0.02 * it_o[k]), (bs, k, infos[k].iterations, it_o[k])
            assert np.linalg.norm(xg[r0:r1] - xo[r0:r1]) <= 1e-8 * np.linalg.norm(xo[r0:r1]), (bs, k)


def test_batched_rejects_column_outside_system(gko, dev):
    B = syn.batched_spd(3, seed=72, n_min=10, n_max=20)
    bad = dict(B)
    bad["col_idx"] = B["col_idx"].copy()
    r1 = B["row_off"][1]
    bad["col_idx"][B["row_ptr"][r1] + 1] = B["row_off"][2] - r1  # one past the second system's size
    with pytest.raises(gko.GkoError) as e:
        gko.Batch(bad)
    assert e.value.status == gko.binding.ERR_INVALID_MATRIX


def test_batched_autotune_and_maxit(gko, dev, orc):
    import torch
    B = syn.batched_spd(200, seed=71)
    G = gko.Batch(B)
    x = torch.zeros(len(B["rhs"]), dtype=torch.float64, device=dev)
    best = G.autotune(_t(B["rhs"], dev), x)
    P, PQ = gko.binding.BATCH_SHARED_P, gko.binding.BATCH_SHARED_PQ
    split = tuple(f | b for f in (P, PQ) for b in (32, 64, 128, 256))
    assert best in (64, 128, 256, 512, 1024, -128, -256, -512, -1024) + split
    assert float(x.abs().max()) == 0.0  # autotune restores x
    s, infos = G.cg(_t(B["rhs"], dev), x, maxit=2)
    assert s == gko.binding.ERR_NOT_CONVERGED
    assert all(i.iterations == 2 for i in infos)


def test_mixed_cg_inner_breakdown_on_indefinite_copy(gko, dev, orc):
    """The BF16 copy of an SPD matrix made indefinite by rounding (see the
    oracle's test of the same case): the inner CG breaks down at its first
    step in every correction, the solve ends NOT_CONVERGED after
    maxit_outer corrections with x unchanged and finite, as the oracle's."""
    import test_oracle as to
    A, b, lo_min, _ = to._indefinite_bf16_case(orc)
    assert lo_min < -1e-4
    _, st_o, o_o, _, res_o = orc.cg_mixed(A, b, prec="bf16", tol=1e-10, maxit_outer=5, inner_tol=1e-1)
    M = gko.Matrix(A)
    x = _t(np.zeros(A["n_rows"]), dev)
    info = M.cg_mixed(_t(b, dev), x, inner="bf16", tol=1e-10, maxit_outer=5, inner_tol=1e-1)
    assert info.status == st_o == gko.binding.ERR_NOT_CONVERGED
    assert info.outer_iterations == o_o == 5 and info.iterations <= 5
    xg = x.cpu().numpy()
    assert np.all(np.isfinite(xg)) and abs(info.rel_residual - res_o) < 1e-12

