"""Restarted GMRES on the GPU against the oracle.  GMRES's residual is the
minimum over the Krylov space, so both sides follow the same curve up to
rounding: parity means both reach the true relative residual, Arnoldi step
counts within max(5, 2 %), the GPU solution's error against the manufactured
solution within 10x of the oracle's, and equal iterates (to rounding) after a
few steps."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("fmt,restart", [("csr", 30), ("ell", 30), ("hybrid", 10), ("coo", 50)])
def test_gmres_convection_diffusion(gko, dev, orc, fmt, restart):
    A = syn.convdiff2d(64, 0.8)
    n = A["n_rows"]
    xt = syn.vector(n, 37)
    b = orc.spmv_csr(A, xt)
    x_o, st_o, it_o, res_o = orc.gmres(A, b, tol=1e-10, restart=restart)
    assert st_o == 0
    M = gko.Matrix(A)
    if fmt != "csr":
        M.convert(fmt)
    x = _t(np.zeros(n), dev)
    info = M.gmres(_t(b, dev), x, tol=1e-10, restart=restart, fmt=fmt)
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert abs(info.iterations - it_o) <= max(5, 0.02 * it_o), (info.iterations, it_o)
    xg = x.cpu().numpy()
    assert orc.true_rel_residual(A, b, xg) <= 1e-10
    e_o = np.linalg.norm(x_o - xt) / np.linalg.norm(xt)
    assert np.linalg.norm(xg - xt) / np.linalg.norm(xt) <= 10 * e_o + 1e-15
    # the same iterate after 7 Arnoldi steps
    x7 = _t(np.zeros(n), dev)
    M.gmres(_t(b, dev), x7, tol=1e-10, restart=restart, maxit=7, fmt=fmt)
    xo7, _, _, _ = orc.gmres(A, b, tol=1e-10, restart=restart, maxit=7)
    assert np.linalg.norm(x7.cpu().numpy() - xo7) <= 1e-10 * np.linalg.norm(xo7)


def _near_identity(n, eps, seed):
    """I + eps R, R a random sparse matrix with entries in [-1, 1)."""
    R = syn.random_csr(n, n, 6, seed=seed)
    rows = np.repeat(np.arange(n), np.diff(R["row_ptr"]))
    D = np.zeros((n, n))
    D[rows, R["col_idx"]] = eps * R["val"]
    D[np.arange(n), np.arange(n)] += 1.0
    r, c = np.nonzero(D)
    return dict(n_rows=n, n_cols=n, row_ptr=np.concatenate([[0], np.cumsum((D != 0).sum(1))]).astype(np.int32),
                col_idx=c.astype(np.int32), val=D[r, c])


def test_gmres_second_pass_precision_paths(gko, dev, orc):
    """The second Gram-Schmidt update runs in FP32 when its coefficients are
    rounding-level against ||w1|| (convection-diffusion: nearly every step)
    and in FP64 when the first pass cancels most of w (A = I + 1e-8 R:
    w = A v_j lies within ~1e-8 of the basis, so the second-pass
    coefficients reach ~1e-16 / 1e-8 of ||w1||, above the 2^-33 bound).
    Both paths match the oracle's FP64 CGS2."""
    A = syn.convdiff2d(64, 0.8)
    n = A["n_rows"]
    b = orc.spmv_csr(A, syn.vector(n, 38))
    M = gko.Matrix(A)
    x = _t(np.zeros(n), dev)
    info = M.gmres(_t(b, dev), x, tol=1e-10, restart=30)
    assert info.status == 0 and info.aux >= 0.9 * info.iterations, (info.aux, info.iterations)
    B = _near_identity(3000, 1e-8, seed=39)
    xt = syn.vector(3000, 40)
    bb = orc.spmv_csr(B, xt)
    x_o, st_o, it_o, _ = orc.gmres(B, bb, tol=1e-13, restart=30)
    MB = gko.Matrix(B)
    x = _t(np.zeros(3000), dev)
    info = MB.gmres(_t(bb, dev), x, tol=1e-13, restart=30)
    assert st_o == 0 and info.status == 0 and abs(info.iterations - it_o) <= 1
    assert info.aux < info.iterations, (info.aux, info.iterations)  # FP64 updates taken
    assert np.linalg.norm(x.cpu().numpy() - x_o) <= 1e-12 * np.linalg.norm(x_o)
    assert orc.true_rel_residual(B, bb, x.cpu().numpy()) <= 1e-13


def test_gmres_three_eigenvalues_and_special_cases(gko, dev, orc):
    blocks = [((1.0, 0.7), (0.0, 2.0)), ((2.0, 0.3), (0.0, 3.0)), ((3.0, -0.5), (0.0, 1.0))]
    nb = 3000
    rp, ci, va = [0], [], []
    for k in range(nb):
        (a, b_), (_, c) = blocks[k % 3]
        r0 = 2 * k
        ci += [r0, r0 + 1]; va += [a, b_]; rp.append(len(ci))
        ci += [r0 + 1]; va += [c]; rp.append(len(ci))
    A = dict(n_rows=2 * nb, n_cols=2 * nb, row_ptr=np.array(rp, np.int32), col_idx=np.array(ci, np.int32),
             val=np.array(va))
    b = syn.vector(2 * nb, 34)
    M = gko.Matrix(A)
    x = _t(np.zeros(2 * nb), dev)
    info = M.gmres(_t(b, dev), x, tol=1e-12, restart=50)
    assert info.status == 0 and info.iterations <= 3, (info.status, info.iterations)
    C = syn.convdiff2d(16, 0.5)
    n = C["n_rows"]
    MC = gko.Matrix(C)
    x = _t(np.ones(n), dev)
    info = MC.gmres(_t(np.zeros(n), dev), x)
    assert info.status == 0 and info.iterations == 0 and float(x.abs().max()) == 0.0
    bc = orc.spmv_csr(C, syn.vector(n, 2))
    x = _t(np.zeros(n), dev)
    info = MC.gmres(_t(bc, dev), x, maxit=3)
    assert info.status == gko.binding.ERR_NOT_CONVERGED and info.iterations == 3
    x = _t(syn.vector(n, 2), dev)
    info = MC.gmres(_t(bc, dev), x)
    assert info.status == 0 and info.iterations == 0
    bn = bc.copy()
    bn[4] = np.nan
    x = _t(np.zeros(n), dev)
    info = MC.gmres(_t(bn, dev), x)
    assert info.status == gko.binding.ERR_BREAKDOWN
