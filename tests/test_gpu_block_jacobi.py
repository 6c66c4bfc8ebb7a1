"""Block-Jacobi preconditioner and block-Jacobi PCG against the oracle.

Block boundaries are integer work: bit-exact.  Inverses come from
Gauss-Jordan elimination on both sides with possibly different pivot
rounding: compared per block against the block's largest inverse entry at
1e-12 (the blocks here are diagonally dominant, condition numbers below
~1e2).  Solver iterates: step counts within max(5, 2 %), the FP64 true
residual confirmed, the solution within 10x the oracle's error."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _from_dense(D):
    r, c = np.nonzero(D)
    return dict(n_rows=D.shape[0], n_cols=D.shape[1],
                row_ptr=np.concatenate([[0], np.cumsum((D != 0).sum(1))]).astype(np.int32),
                col_idx=c.astype(np.int32), val=D[r, c])


def _dominant(A, shift):
    """A + shift * I (diagonal stored for every row)."""
    n = A["n_rows"]
    rows = np.repeat(np.arange(n), np.diff(A["row_ptr"]))
    r = np.concatenate([rows, np.arange(n)])
    c = np.concatenate([A["col_idx"].astype(np.int64), np.arange(n)])
    v = np.concatenate([A["val"], np.full(n, float(shift))])
    key = r * n + c
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    uk, start = np.unique(key, return_index=True)
    vs = np.add.reduceat(v, start)
    ur, uc = uk // n, uk % n
    return dict(n_rows=n, n_cols=n, row_ptr=np.concatenate([[0], np.cumsum(np.bincount(ur, minlength=n))]).astype(np.int32),
                col_idx=uc.astype(np.int32), val=vs)


def _supervariable_matrix(nx=10, dof=3, seed=41):
    """2-D 5-point pattern with `dof` unknowns per grid point (each row of a
    point has the same column list: supervariables of `dof` rows),
    nonsymmetric values, diagonally dominant."""
    L = syn.laplace2d(nx)
    n0 = L["n_rows"]
    D0 = np.zeros((n0, n0))
    rows = np.repeat(np.arange(n0), np.diff(L["row_ptr"]))
    D0[rows, L["col_idx"]] = 1.0
    P = np.kron(D0, np.ones((dof, dof)))
    n = n0 * dof
    V = syn.uniform_pm1(seed, 1, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    D = np.where(P != 0, V, 0.0)
    D[np.arange(n), np.arange(n)] = 6.0 * dof
    return _from_dense(D)


def mats():
    return {
        "laplace2d_20": syn.laplace2d(20),
        "diffusion7_10": syn.diffusion7(10, 1.0, seed=6),
        "supervariables_3": _supervariable_matrix(),
        "random_nonsym": _dominant(syn.random_csr(2000, 2000, 9, seed=42), 12.0),
        "blockdiag_8": _dominant(syn.block_diagonal(800, 8, seed=43), 10.0),
        "one_row": _dominant(syn.random_csr(1, 1, 1, seed=44), 3.0),
    }


@pytest.mark.parametrize("bs", [1, 3, 8, 13, 32])
def test_blocks_inverses_and_apply_match_oracle(gko, dev, orc, bs):
    import torch
    for name, A in mats().items():
        n = A["n_rows"]
        M = gko.Matrix(A)
        P = gko.BlockJacobi(M, bs)
        bp, inv = P.export()
        bp_o = orc.bj_blocks(A, bs)
        assert np.array_equal(bp, bp_o), (name, bs)
        st, inv_o = orc.bj_invert(A, bp_o, bs)
        assert st == orc.OK
        for o, e in zip(bp_o[:-1], bp_o[1:]):
            s = e - o
            seg = slice(o * bs, o * bs + s * s)
            scale = np.abs(inv_o[seg]).max()
            assert np.all(np.abs(inv[seg] - inv_o[seg]) <= 1e-12 * scale), (name, bs, o)
            assert np.all(inv[o * bs + s * s:(o + s) * bs] == 0.0)  # unused slots stay zero
        r = syn.vector(n, 45)
        z = torch.empty(n, dtype=torch.float64, device=dev)
        P.apply(_t(r, dev), z)
        torch.cuda.synchronize()
        z_o = orc.bj_apply(bp_o, bs, inv_o, r)
        # magnitude of the terms of each z_i
        mag = orc.bj_apply(bp_o, bs, np.abs(inv_o), np.abs(r))
        assert np.all(np.abs(z.cpu().numpy() - z_o) <= 1e-12 * mag + 1e-300), (name, bs)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo"])
def test_pcg_block_jacobi_matches_oracle(gko, dev, orc, fmt):
    A = syn.diffusion7(24, 1.0, seed=6)
    n = A["n_rows"]
    xt = syn.vector(n, 46)
    b = orc.spmv_csr(A, xt)
    M = gko.Matrix(A)
    if fmt != "csr":
        M.convert(fmt)
    for bs in (4, 24):
        x_o, st_o, it_o, res_o = orc.pcg_block_jacobi(A, b, bs, tol=1e-10, maxit=5000)
        assert st_o == orc.OK
        P = gko.BlockJacobi(M, bs)
        x = _t(np.zeros(n), dev)
        info = M.pcg_block_jacobi(P, _t(b, dev), x, tol=1e-10, maxit=5000, fmt=fmt)
        assert info.status == 0 and info.rel_residual <= 1e-10
        assert abs(info.iterations - it_o) <= max(5, 0.02 * it_o), (bs, info.iterations, it_o)
        xg = x.cpu().numpy()
        assert orc.true_rel_residual(A, b, xg) <= 1e-10
        e_o = np.linalg.norm(x_o - xt) / np.linalg.norm(xt)
        assert np.linalg.norm(xg - xt) / np.linalg.norm(xt) <= 10 * e_o + 1e-15
    # larger blocks along x take fewer steps than point Jacobi
    x = _t(np.zeros(n), dev)
    it_j = M.pcg_jacobi(_t(b, dev), x, tol=1e-10, fmt=fmt).iterations
    assert info.iterations < it_j


def test_pcg_block_jacobi_fixed_steps_match_oracle(gko, dev, orc):
    """After k steps (tol = 0: no early stop) the iterates agree with the
    oracle's to rounding."""
    A = _supervariable_matrix(12, 3, seed=47)
    # symmetric positive definite version: (A + A^T)/2 keeps the pattern
    D = np.zeros((A["n_rows"],) * 2)
    rows = np.repeat(np.arange(A["n_rows"]), np.diff(A["row_ptr"]))
    D[rows, A["col_idx"]] = A["val"]
    S = _from_dense(0.5 * (D + D.T))
    n = S["n_rows"]
    b = orc.spmv_csr(S, syn.vector(n, 48))
    M = gko.Matrix(S)
    P = gko.BlockJacobi(M, 6)
    for k in (1, 3, 10):
        x_o, _, it_o, _ = orc.pcg_block_jacobi(S, b, 6, tol=0.0, maxit=k)
        x = _t(np.zeros(n), dev)
        info = M.pcg_block_jacobi(P, _t(b, dev), x, tol=0.0, maxit=k)
        assert info.iterations == it_o == k
        assert np.linalg.norm(x.cpu().numpy() - x_o) <= 1e-12 * np.linalg.norm(x_o)


def test_block_jacobi_special_cases(gko, dev, orc):
    A = syn.laplace2d(16)
    n = A["n_rows"]
    M = gko.Matrix(A)
    P = gko.BlockJacobi(M, 8)
    x = _t(np.ones(n), dev)
    info = M.pcg_block_jacobi(P, _t(np.zeros(n), dev), x)
    assert info.status == 0 and info.iterations == 0 and float(x.abs().max()) == 0.0
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x = _t(np.zeros(n), dev)
    info = M.pcg_block_jacobi(P, _t(b, dev), x, maxit=3)
    assert info.status == gko.binding.ERR_NOT_CONVERGED and info.iterations == 3
    # exact preconditioner: A block-diagonal with the detected blocks, one step
    B = _dominant(syn.block_diagonal(256, 8, seed=49), 10.0)
    Dd = np.zeros((256, 256))
    rows = np.repeat(np.arange(256), np.diff(B["row_ptr"]))
    Dd[rows, B["col_idx"]] = B["val"]
    S = _from_dense(Dd @ Dd.T)  # SPD, same 8 x 8 block pattern
    MS = gko.Matrix(S)
    xt = syn.vector(256, 50)
    bS = orc.spmv_csr(S, xt)
    x = _t(np.zeros(256), dev)
    info = MS.pcg_block_jacobi(gko.BlockJacobi(MS, 8), _t(bS, dev), x, tol=1e-12)
    assert info.status == 0 and info.iterations == 1
    assert np.linalg.norm(x.cpu().numpy() - xt) <= 1e-12 * np.linalg.norm(xt)
    # a zero row makes its block singular: refused at creation
    Z = dict(A)
    Z["val"] = A["val"].copy()
    Z["val"][A["row_ptr"][5]:A["row_ptr"][6]] = 0.0
    with pytest.raises(gko.GkoError) as e:
        gko.BlockJacobi(gko.Matrix(Z), 4)
    assert e.value.status == gko.binding.ERR_BREAKDOWN
    # invalid sizes and a preconditioner of another matrix
    for bad in (0, 33):
        with pytest.raises(gko.GkoError) as e:
            gko.BlockJacobi(M, bad)
        assert e.value.status == gko.binding.ERR_INVALID_ARG
    other = gko.BlockJacobi(gko.Matrix(syn.laplace2d(8)), 4)
    with pytest.raises(gko.GkoError) as e:
        M.pcg_block_jacobi(other, _t(b, dev), _t(np.zeros(n), dev))
    assert e.value.status == gko.binding.ERR_DIM_MISMATCH
    # non-square matrices are refused
    with pytest.raises(gko.GkoError) as e:
        gko.BlockJacobi(gko.Matrix(syn.random_csr(10, 12, 3, seed=51)), 4)
    assert e.value.status == gko.binding.ERR_DIM_MISMATCH


def test_full_size_generation_sampled(gko, dev, orc):
    """The 7-point 160^3 operator with 8-row blocks (the benchmark's
    preconditioner): all block boundaries bit-exact, the inverses of 2,000
    sampled blocks against the oracle's."""
    A = syn.diffusion7(160, 1.0, seed=6)
    n = A["n_rows"]
    M = gko.Matrix(A)
    P = gko.BlockJacobi(M, 8)
    bp, inv = P.export()
    bp_o = orc.bj_blocks(A, 8)
    assert np.array_equal(bp, bp_o)
    st, inv_o = orc.bj_invert(A, bp_o, 8)
    assert st == orc.OK
    rng = np.random.default_rng(52)
    for k in rng.choice(len(bp_o) - 1, size=2000, replace=False):
        o, s = bp_o[k], bp_o[k + 1] - bp_o[k]
        seg = slice(o * 8, o * 8 + s * s)
        assert np.all(np.abs(inv[seg] - inv_o[seg]) <= 1e-12 * np.abs(inv_o[seg]).max()), k
    assert n == bp[-1]
