"""CG for several right-hand sides (gko_cg_multi) against the oracle's CG
applied column by column: each column is its own Hestenes-Stiefel
recurrence, so its step count must match the single-right-hand-side oracle
within max(5, 2 %), its true residual must meet the tolerance and its
solution must be within 10x the oracle's error of the manufactured one."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _block(A, k, seed):
    """k manufactured solutions of different smoothness, their right-hand
    sides, and one zero column when k > 2."""
    import oracle as orc
    n = A["n_rows"]
    Xt = np.zeros((n, k))
    for c in range(k):
        v = syn.vector(n, seed + c)
        if c % 3 == 1:  # smooth columns converge sooner
            v = np.cumsum(v) / np.sqrt(n)
        Xt[:, c] = v
    if k > 2:
        Xt[:, 2] = 0.0
    Bm = np.stack([orc.spmv_csr(A, Xt[:, c]) for c in range(k)], axis=1)
    return Xt, Bm


@pytest.mark.parametrize("k", [1, 3, 8, 13])
def test_cg_multi_matches_single_rhs_oracle(gko, dev, orc, k):
    A = syn.diffusion7(16, 1.0, seed=6)
    n = A["n_rows"]
    Xt, Bm = _block(A, k, 60)
    M = gko.Matrix(A)
    X = _t(np.zeros((n, k)), dev)
    s, infos = M.cg_multi(_t(Bm, dev), X, tol=1e-10, maxit=5000)
    assert s == 0
    Xg = X.cpu().numpy()
    for c in range(k):
        info = infos[c]
        if not Bm[:, c].any():
            assert info.iterations == 0 and info.status == 0 and not Xg[:, c].any()
            continue
        x_o, st_o, it_o, _ = orc.cg(A, Bm[:, c], tol=1e-10, maxit=5000)
        assert st_o == 0 and info.status == 0 and info.rel_residual <= 1e-10, c
        assert abs(info.iterations - it_o) <= max(5, 0.02 * it_o), (c, info.iterations, it_o)
        assert orc.true_rel_residual(A, Bm[:, c], Xg[:, c]) <= 1e-10
        e_o = np.linalg.norm(x_o - Xt[:, c]) / np.linalg.norm(Xt[:, c])
        assert np.linalg.norm(Xg[:, c] - Xt[:, c]) / np.linalg.norm(Xt[:, c]) <= 10 * e_o + 1e-15
    if k > 2:  # columns stop at their own step counts
        its = [infos[c].iterations for c in range(k) if Bm[:, c].any()]
        assert max(its) > min(its)


def test_cg_multi_strided_blocks_and_initial_guess(gko, dev, orc):
    """B and X as column slices of wider blocks (ldb, ldx > k); a column
    whose initial guess is already the solution takes no step."""
    import torch
    A = syn.laplace2d(48)
    n = A["n_rows"]
    Xt, Bm = _block(A, 5, 70)
    Bw = torch.zeros((n, 9), dtype=torch.float64, device=dev)
    Xw = torch.zeros((n, 11), dtype=torch.float64, device=dev)
    Bw[:, 2:7] = _t(Bm, dev)
    Xw[:, 1:6] = 0.0
    Xw[:, 1 + 3] = _t(Xt[:, 3], dev)  # column 3 starts at its solution
    M = gko.Matrix(A)
    s, infos = M.cg_multi(Bw[:, 2:7], Xw[:, 1:6], tol=1e-10)
    assert s == 0
    assert infos[3].iterations == 0
    Xg = Xw.cpu().numpy()
    assert not Xg[:, 0].any() and not Xg[:, 6:].any()  # outside the slice untouched
    for c in range(5):
        if Bm[:, c].any():
            assert orc.true_rel_residual(A, Bm[:, c], Xg[:, 1 + c]) <= 1e-10
    # each column's iterates equal the single-vector CG's after a few steps
    for c in (0, 1):
        x1 = _t(np.zeros(n), dev)
        M.cg(_t(Bm[:, c], dev), x1, tol=1e-10, maxit=7)
        X7 = torch.zeros((n, 5), dtype=torch.float64, device=dev)
        M.cg_multi(_t(Bm, dev), X7, tol=1e-10, maxit=7)
        assert torch.linalg.vector_norm(X7[:, c] - x1) <= 1e-10 * torch.linalg.vector_norm(x1)


def test_cg_multi_maxit_breakdown_and_errors(gko, dev, orc):
    import torch
    A = syn.laplace2d(32)
    n = A["n_rows"]
    _, Bm = _block(A, 4, 80)
    M = gko.Matrix(A)
    X = torch.zeros((n, 4), dtype=torch.float64, device=dev)
    s, infos = M.cg_multi(_t(Bm, dev), X, maxit=3)
    assert s == gko.binding.ERR_NOT_CONVERGED
    for c in range(4):
        if Bm[:, c].any():
            assert infos[c].iterations == 3 and infos[c].status == gko.binding.ERR_NOT_CONVERGED
    N = dict(A)
    N["val"] = -A["val"]  # negative definite: every column breaks down at its first step
    X = torch.zeros((n, 4), dtype=torch.float64, device=dev)
    s, infos = gko.Matrix(N).cg_multi(_t(Bm, dev), X)
    assert s == gko.binding.ERR_BREAKDOWN
    assert all(infos[c].status == gko.binding.ERR_BREAKDOWN for c in range(4) if Bm[:, c].any())
    assert bool(torch.isfinite(X).all())
    for bad_k in (0, 33):
        Bk = torch.zeros((n, max(bad_k, 1)), dtype=torch.float64, device=dev)[:, :bad_k]
        with pytest.raises(gko.GkoError) as e:
            gko.binding.gko_cg_multi(M.handle, bad_k, Bk.data_ptr(), max(bad_k, 1), Bk.data_ptr(), max(bad_k, 1),
                                     1e-10, 100, 0)
        assert e.value.status == gko.binding.ERR_INVALID_ARG
    with pytest.raises(gko.GkoError) as e:
        gko.binding.gko_cg_multi(M.handle, 4, X.data_ptr(), 3, X.data_ptr(), 4, 1e-10, 100, 0)
    assert e.value.status == gko.binding.ERR_INVALID_ARG
