"""Pins of the CPU oracle against facts that do not come from the oracle itself:
dense brute force, closed forms of the 5-point Laplacian, exact rational
arithmetic, a textbook dense solver, exhaustive enumeration and finite
differences.  Each pin is chosen so that a plausible slip in the oracle (a
dropped term, a wrong index, a transposed operand) fails it."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn


def small_mats():
    out = []
    for seed, (n, m, k, e) in enumerate([(1, 1, 1, 0.0), (7, 5, 5, 0.3), (33, 40, 9, 0.2),
                                         (64, 64, 20, 0.1), (65, 17, 17, 0.5), (50, 80, 0, 0.0),
                                         (96, 96, 31, 0.05)]):
        out.append(syn.random_csr(n, m, k, seed=100 + seed, empty_frac=e))
    return out


def dense(A):
    D = np.zeros((A["n_rows"], A["n_cols"]))
    rp = A["row_ptr"]
    for i in range(A["n_rows"]):
        for k in range(rp[i], rp[i + 1]):
            D[i, A["col_idx"][k]] += A["val"][k]
    return D


# ---------------------------------------------------------------- SpMV pins

@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0), (2.5, -0.5), (0.0, 2.0)])
def test_every_format_matches_dense_matvec(orc, alpha, beta):
    for A in small_mats():
        n, m = A["n_rows"], A["n_cols"]
        x = syn.vector(m, 5)
        y0 = syn.vector(n, 6)
        ref = alpha * (dense(A) @ x) + beta * y0
        mag = abs(alpha) * (np.abs(dense(A)) @ np.abs(x)) + abs(beta) * np.abs(y0)
        tol = 1e-14 * mag + 1e-300
        outs = {
            "csr": orc.spmv_csr(A, x, alpha, beta, y0),
            "coo": orc.spmv_coo(n, orc.to_coo(A), x, alpha, beta, y0),
            "ell": orc.spmv_ell(n, orc.to_ell(A), x, alpha, beta, y0),
            "sellp32": orc.spmv_sellp(n, orc.to_sellp(A, 32), x, alpha, beta, y0),
            "sellp64f4": orc.spmv_sellp(n, orc.to_sellp(A, 64, 4), x, alpha, beta, y0),
            "hybrid": orc.spmv_hybrid(n, orc.to_hybrid(A), x, alpha, beta, y0),
            "hybrid_k1": orc.spmv_hybrid(n, orc.to_hybrid(A, K=1), x, alpha, beta, y0),
        }
        for name, y in outs.items():
            assert np.all(np.abs(y - ref) <= tol), (name, n, m)


def test_beta_zero_does_not_read_y(orc):
    A = small_mats()[3]
    x = syn.vector(A["n_cols"], 1)
    y = np.full(A["n_rows"], np.nan)
    out = orc.spmv_csr(A, x, 1.0, 0.0, y)
    assert np.all(np.isfinite(out))


def test_integer_values_make_every_format_exact(orc):
    """Integer-valued A and x: every partial sum is an exactly representable
    integer, so each format equals the exact integer product bit for bit."""
    for A in small_mats() + [syn.powerlaw(3000, 20.0, 1.5, 400, seed=9)]:
        A = dict(A)
        A["val"] = np.round(A["val"] * 8.0)
        n, m = A["n_rows"], A["n_cols"]
        xi = np.round(syn.vector(m, 3) * 16.0)
        exact = np.zeros(n, dtype=np.int64)
        rp = A["row_ptr"]
        for i in range(n):
            for k in range(rp[i], rp[i + 1]):
                exact[i] += int(A["val"][k]) * int(xi[A["col_idx"][k]])
        ys = [orc.spmv_csr(A, xi), orc.spmv_coo(n, orc.to_coo(A), xi),
              orc.spmv_sellp(n, orc.to_sellp(A, 64), xi), orc.spmv_hybrid(n, orc.to_hybrid(A), xi)]
        if orc.max_row_len(A) <= 64:
            ys.append(orc.spmv_ell(n, orc.to_ell(A), xi))
        for y in ys:
            assert np.array_equal(y, exact.astype(np.float64))


def test_laplacian_row_sums_closed_form(orc):
    """A * 1 for the 5-point Dirichlet Laplacian: 0 inside, 1 on an edge, 2 at a corner."""
    nx = 128
    A = syn.laplace2d(nx)
    y = orc.spmv_csr(A, np.ones(nx * nx))
    idx = np.arange(nx * nx)
    i, j = idx % nx, idx // nx
    boundary_sides = (i == 0).astype(int) + (i == nx - 1) + (j == 0) + (j == nx - 1)
    assert np.array_equal(y, boundary_sides.astype(np.float64))
    assert A["row_ptr"][-1] == 5 * nx * nx - 4 * nx


@pytest.mark.parametrize("jk", [(1, 1), (3, 7), (64, 2), (127, 127), (100, 33)])
def test_laplacian_eigenpairs(orc, jk):
    """v(p,q) = sin(j p pi/(nx+1)) sin(k q pi/(nx+1)), lambda = 4 - 2cos(j pi/(nx+1)) - 2cos(k pi/(nx+1))."""
    nx = 128
    jj, kk = jk
    A = syn.laplace2d(nx)
    idx = np.arange(nx * nx)
    p, q = idx % nx + 1, idx // nx + 1
    v = np.sin(jj * p * np.pi / (nx + 1)) * np.sin(kk * q * np.pi / (nx + 1))
    lam = 4 - 2 * math.cos(jj * math.pi / (nx + 1)) - 2 * math.cos(kk * math.pi / (nx + 1))
    Av = orc.spmv_csr(A, v)
    assert np.linalg.norm(Av - lam * v) <= 1e-13 * np.linalg.norm(v)


def test_dot2_matches_exact_rational_sum(orc):
    rng = np.random.default_rng(0)
    for n in (1, 10, 1000):
        a = rng.standard_normal(n) * 10.0 ** rng.integers(-8, 8, n)
        b = rng.standard_normal(n)
        exact = sum(Fraction(float(u)) * Fraction(float(w)) for u, w in zip(a, b))
        d2 = orc.dot2(a, b)
        mag = float(np.sum(np.abs(a * b)))
        assert abs(Fraction(d2) - exact) <= Fraction(2.0 ** -52) * abs(exact) + Fraction(mag * 2.0 ** -100)
        # and the plain dot is the sequential definition
        s = 0.0
        for u, w in zip(a, b):
            s = s + u * w
        assert orc.dot(a, b) == s


def test_spmv_dot2_reference_is_near_exact(orc):
    A = syn.powerlaw(2000, 20.0, 1.5, 2000, seed=11)
    x = syn.vector(2000, 12)
    y0 = syn.vector(2000, 13)
    yref, mag = orc.spmv_dot2(A, x, 1.5, -0.25, y0)
    rp = A["row_ptr"]
    for i in range(0, 2000, 97):
        ex = Fraction(1.5) * sum(Fraction(float(A["val"][k])) * Fraction(float(x[A["col_idx"][k]]))
                                 for k in range(rp[i], rp[i + 1])) + Fraction(-0.25) * Fraction(float(y0[i]))
        assert abs(Fraction(float(yref[i])) - ex) <= Fraction(2.0 ** -52) * abs(ex) + Fraction(float(mag[i]) * 2.0 ** -104)
        m_ex = 1.5 * sum(abs(A["val"][k] * x[A["col_idx"][k]]) for k in range(rp[i], rp[i + 1])) + 0.25 * abs(y0[i])
        assert abs(mag[i] - m_ex) <= 1e-13 * m_ex


# ---------------------------------------------------------- format layouts

def test_round_trips_are_bit_exact(orc):
    mats = small_mats() + [syn.powerlaw(5000, 20.0, 1.5, 3000, seed=21), syn.laplace2d(20)]
    for A in mats:
        A = dict(A)
        A["val"] = A["val"].copy()
        if len(A["val"]) > 3:
            A["val"][::3] = 0.0  # explicit stored zeros must survive
            A["val"][1::7] = -0.0
        n, m = A["n_rows"], A["n_cols"]
        back = [orc.coo_to_csr(n, orc.to_coo(A), m),
                orc.sellp_to_csr(n, orc.to_sellp(A, 32), m),
                orc.sellp_to_csr(n, orc.to_sellp(A, 64, 8), m),
                orc.hybrid_to_csr(n, orc.to_hybrid(A), m),
                orc.hybrid_to_csr(n, orc.to_hybrid(A, K=0), m),
                orc.hybrid_to_csr(n, orc.to_hybrid(A, K=3), m)]
        if orc.max_row_len(A) <= 64:
            back.append(orc.ell_to_csr(n, orc.to_ell(A), m))
        for B in back:
            assert np.array_equal(B["row_ptr"], A["row_ptr"])
            assert np.array_equal(B["col_idx"], A["col_idx"])
            assert B["val"].tobytes() == A["val"].tobytes()


def test_ell_layout_brute_force(orc):
    A = small_mats()[2]
    E = orc.to_ell(A)
    n = A["n_rows"]
    assert E["n_pad"] == 64 and E["K"] == int(np.diff(A["row_ptr"]).max())
    col = E["col"].reshape(E["K"], E["n_pad"])
    val = E["val"].reshape(E["K"], E["n_pad"])
    for i in range(E["n_pad"]):
        L = A["row_ptr"][i + 1] - A["row_ptr"][i] if i < n else 0
        for k in range(E["K"]):
            if k < L:
                assert col[k, i] == A["col_idx"][A["row_ptr"][i] + k]
                assert val[k, i] == A["val"][A["row_ptr"][i] + k]
            else:
                assert col[k, i] == -1 and val[k, i] == 0.0 and not np.signbit(val[k, i])


def test_sellp_layout_brute_force(orc):
    A = syn.random_csr(150, 150, 12, seed=31, empty_frac=0.2)
    for S, f in ((32, 1), (64, 1), (32, 4)):
        s = orc.to_sellp(A, S, f)
        L = np.diff(A["row_ptr"])
        ns = -(-150 // S)
        acc = 0
        for t in range(ns):
            w = int(L[t * S:(t + 1) * S].max())
            w = -(-w // f) * f
            assert s["slice_len"][t] == w and s["slice_set"][t] == acc
            acc += w
        assert s["slice_set"][ns] == acc and len(s["col"]) == acc * S
        for i in range(150):
            t, l = divmod(i, S)
            for k in range(s["slice_len"][t]):
                slot = (s["slice_set"][t] + k) * S + l
                if k < L[i]:
                    assert s["col"][slot] == A["col_idx"][A["row_ptr"][i] + k]
                else:
                    assert s["col"][slot] == -1


def test_hybrid_width_is_byte_argmin(orc):
    for A in small_mats() + [syn.powerlaw(4000, 20.0, 1.5, 2000, seed=41)]:
        L = np.diff(A["row_ptr"]).astype(np.int64)
        n_pad = -(-A["n_rows"] // 32) * 32
        for s_v in (8, 4, 2):
            costs = [n_pad * K * (s_v + 4) + int(np.maximum(L - K, 0).sum()) * (s_v + 8)
                     for K in range(int(L.max(initial=0)) + 1)]
            assert orc.hybrid_width(A, s_v) == int(np.argmin(costs))


# ----------------------------------------------------------------- solvers

def test_cholesky_matches_numpy(orc):
    rng = np.random.default_rng(3)
    for n in (1, 5, 40):
        G = rng.standard_normal((n, n))
        A = G @ G.T + n * np.eye(n)
        b = rng.standard_normal(n)
        x, st = orc.cholesky_solve(A, b)
        assert st == 0
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)
    x, st = orc.cholesky_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2))
    assert st == orc.BREAKDOWN


def test_cg_manufactured_solution_laplace(orc):
    A = syn.laplace2d(128)
    n = A["n_rows"]
    xt = syn.vector(n, 1)
    b = orc.spmv_csr(A, xt)
    x, st, it, res = orc.cg(A, b, tol=1e-10)
    assert st == orc.OK and res <= 1e-10
    assert 350 <= it <= 420
    lam_min = 4 - 4 * math.cos(math.pi / 129)
    lam_max = 4 + 4 * math.cos(math.pi / 129)
    kappa = lam_max / lam_min
    assert 6700 < kappa < 6800
    assert np.linalg.norm(x - xt) <= kappa * 1e-10 * np.linalg.norm(xt)


def test_cg_small_spd_vs_cholesky(orc):
    B = syn.batched_spd(6, seed=5, n_min=8, n_max=60)
    for s in range(6):
        r0, r1 = B["row_off"][s], B["row_off"][s + 1]
        k0, k1 = B["row_ptr"][r0], B["row_ptr"][r1]
        A = dict(n_rows=r1 - r0, n_cols=r1 - r0, row_ptr=B["row_ptr"][r0:r1 + 1] - k0,
                 col_idx=B["col_idx"][k0:k1], val=B["val"][k0:k1])
        D = dense(A)
        assert np.array_equal(D, D.T)
        b = B["rhs"][r0:r1]
        xc, st = orc.cholesky_solve(D, b)
        assert st == 0
        x, st, it, res = orc.cg(A, b, tol=1e-12)
        assert st == orc.OK
        assert np.linalg.norm(x - xc) <= 1e-10 * np.linalg.norm(xc)
        assert it <= r1 - r0 + 5


def test_cg_special_cases(orc):
    A = syn.laplace2d(8)
    n = A["n_rows"]
    x, st, it, res = orc.cg(A, np.zeros(n), x0=np.ones(n))
    assert st == orc.OK and it == 0 and np.all(x == 0)
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x, st, it, res = orc.cg(A, b, maxit=1)
    assert st == orc.NOT_CONVERGED and it == 1
    Aneg = dict(A)
    Aneg["val"] = -A["val"]
    x, st, it, res = orc.cg(Aneg, b)
    assert st == orc.BREAKDOWN
    # an exact initial guess needs no iteration
    xt = syn.vector(n, 2)
    x, st, it, res = orc.cg(A, b, x0=xt)
    assert st == orc.OK and it == 0


def test_cg_matches_scipy_solution(orc):
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    A = syn.diffusion7(12, 1.0, seed=6)
    n = A["n_rows"]
    M = sp.csr_matrix((A["val"], A["col_idx"], A["row_ptr"]), shape=(n, n))
    b = syn.vector(n, 4)
    x, st, it, res = orc.cg(A, b, tol=1e-12)
    xs = spl.spsolve(M.tocsc(), b)
    assert st == orc.OK
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def _diag_spd(eigs):
    n = len(eigs)
    return dict(n_rows=n, n_cols=n, row_ptr=np.arange(n + 1, dtype=np.int32),
                col_idx=np.arange(n, dtype=np.int32), val=np.asarray(eigs, dtype=np.float64))


@pytest.mark.parametrize("solver", ["cg", "cg_single_reduction"])
def test_cg_first_step_is_steepest_descent(orc, solver):
    """From x0 = 0 the first CG iterate is the exact line minimum along b:
    x1 = (b.b / b.Ab) b (closed form of one step of either form)."""
    A = syn.diffusion7(6, 1.0, seed=3)
    n = A["n_rows"]
    b = syn.vector(n, 11)
    D = dense(A)
    x1 = (b @ b) / (b @ (D @ b)) * b
    x, st, it, res = getattr(orc, solver)(A, b, maxit=1)
    assert it == 1
    assert np.linalg.norm(x - x1) <= 1e-14 * np.linalg.norm(x1)


@pytest.mark.parametrize("solver", ["cg", "cg_single_reduction"])
def test_cg_finite_termination(orc, solver):
    """CG on an SPD matrix with m distinct eigenvalues reaches the solution
    in at most m steps (exact arithmetic; a well-conditioned case in FP64)."""
    eigs = np.repeat([1.0, 1.5, 2.25, 3.0, 4.0], 7)
    A = _diag_spd(eigs)
    b = syn.vector(len(eigs), 12)
    x, st, it, res = getattr(orc, solver)(A, b, tol=1e-13)
    assert st == orc.OK and it <= 5
    assert np.allclose(x, b / eigs, rtol=1e-12, atol=0)
    # one step short of m leaves a residual far above the tolerance
    x, st, it, res = getattr(orc, solver)(A, b, tol=1e-13, maxit=4)
    assert st == orc.NOT_CONVERGED and res > 1e-6


def test_cg_single_reduction_matches_hestenes_stiefel(orc):
    """The two forms produce the same iterates up to rounding: same step
    counts on the 5-point Laplacian and solutions within the CG error bound
    of the manufactured solution."""
    A = syn.laplace2d(64)
    n = A["n_rows"]
    xt = syn.vector(n, 1)
    b = orc.spmv_csr(A, xt)
    x0, st0, it0, res0 = orc.cg(A, b, tol=1e-10)
    x1, st1, it1, res1 = orc.cg_single_reduction(A, b, tol=1e-10)
    assert st0 == st1 == orc.OK and res1 <= 1e-10
    assert abs(it0 - it1) <= 2
    for k in (3, 17, 40):  # the same iterate after k steps
        xa, _, _, _ = orc.cg(A, b, maxit=k)
        xb, _, _, _ = orc.cg_single_reduction(A, b, maxit=k)
        assert np.linalg.norm(xa - xb) <= 1e-10 * np.linalg.norm(xa)


def test_cg_single_reduction_special_cases(orc):
    A = syn.laplace2d(8)
    n = A["n_rows"]
    x, st, it, res = orc.cg_single_reduction(A, np.zeros(n), x0=np.ones(n))
    assert st == orc.OK and it == 0 and np.all(x == 0)
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x, st, it, res = orc.cg_single_reduction(A, b, maxit=1)
    assert st == orc.NOT_CONVERGED and it == 1
    Aneg = dict(A)
    Aneg["val"] = -A["val"]
    x, st, it, res = orc.cg_single_reduction(Aneg, b)
    assert st == orc.BREAKDOWN
    x, st, it, res = orc.cg_single_reduction(A, b, x0=syn.vector(n, 2))
    assert st == orc.OK and it == 0


def _scaled(A, s):
    """D A D for the diagonal scaling s (SPD stays SPD)."""
    rows = np.repeat(np.arange(A["n_rows"]), np.diff(A["row_ptr"]))
    B = dict(A)
    B["val"] = A["val"] * s[rows] * s[A["col_idx"]]
    return B


def test_pcg_jacobi_diagonal_matrix_one_step(orc):
    """M = A when A is diagonal: the preconditioned system is the identity
    and one step gives the exact solution."""
    eigs = 1.0 + np.arange(40) * 0.37
    A = _diag_spd(eigs)
    b = syn.vector(40, 21)
    x, st, it, res = orc.pcg_jacobi(A, b, tol=1e-14)
    assert st == orc.OK and it == 1
    assert np.allclose(x, b / eigs, rtol=1e-15, atol=0)


def test_pcg_jacobi_constant_diagonal_equals_cg(orc):
    """A constant diagonal makes D^-1 a multiple of the identity: the
    iterates are those of plain CG (same steps, same solution)."""
    A = syn.laplace2d(48)
    n = A["n_rows"]
    b = orc.spmv_csr(A, syn.vector(n, 22))
    for k in (1, 5, 30):
        xa, _, _, _ = orc.cg(A, b, maxit=k)
        xb, _, _, _ = orc.pcg_jacobi(A, b, maxit=k)
        assert np.linalg.norm(xa - xb) <= 1e-11 * np.linalg.norm(xa)
    _, s0, i0, _ = orc.cg(A, b, tol=1e-10)
    _, s1, i1, r1 = orc.pcg_jacobi(A, b, tol=1e-10)
    assert s0 == s1 == orc.OK and abs(i0 - i1) <= 1 and r1 <= 1e-10


def test_pcg_jacobi_removes_bad_row_scaling(orc):
    """On D A D with a wildly varying D, Jacobi PCG needs about the steps
    of A itself while plain CG needs many more; both reach the manufactured
    solution."""
    A0 = syn.laplace2d(32)
    n = A0["n_rows"]
    s = 10.0 ** (3.0 * syn.uniform01(23, 1, np.arange(n, dtype=np.uint64)))
    A = _scaled(A0, s)
    xt = syn.vector(n, 24)
    b = orc.spmv_csr(A, xt)
    xc, sc, ic, rc = orc.cg(A, b, tol=1e-10, maxit=20000)
    xp, sp, ip, rp = orc.pcg_jacobi(A, b, tol=1e-10, maxit=20000)
    _, _, i0, _ = orc.cg(A0, orc.spmv_csr(A0, xt), tol=1e-10)
    assert sp == orc.OK and rp <= 1e-10
    assert ip <= 1.5 * i0 + 10 and ic > 3 * ip
    assert np.linalg.norm(xp - xt) <= 1e-5 * np.linalg.norm(xt)


def test_pcg_jacobi_special_cases(orc):
    A = syn.laplace2d(8)
    n = A["n_rows"]
    x, st, it, res = orc.pcg_jacobi(A, np.zeros(n), x0=np.ones(n))
    assert st == orc.OK and it == 0 and np.all(x == 0)
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x, st, it, res = orc.pcg_jacobi(A, b, maxit=2)
    assert st == orc.NOT_CONVERGED and it == 2
    Z = dict(A)
    Z["val"] = np.where(A["col_idx"] == np.repeat(np.arange(n), np.diff(A["row_ptr"])), 0.0, A["val"])
    x, st, it, res = orc.pcg_jacobi(Z, b)
    assert st == orc.BREAKDOWN and it == 0


def _csr_rows(n, rows):
    """CSR dict from a list of (column list, value list) per row."""
    L = [len(c) for c, _ in rows]
    return dict(n_rows=n, n_cols=n, row_ptr=np.concatenate([[0], np.cumsum(L)]).astype(np.int32),
                col_idx=np.array([c for cs, _ in rows for c in cs], dtype=np.int32),
                val=np.array([v for _, vs in rows for v in vs], dtype=np.float64))


def _laplace1d(n):
    rows = []
    for i in range(n):
        cs = [j for j in (i - 1, i, i + 1) if 0 <= j < n]
        rows.append((cs, [2.0 if j == i else -1.0 for j in cs]))
    return _csr_rows(n, rows)


@pytest.mark.parametrize("max_bs,want", [(4, [0, 4, 8, 10]), (32, [0, 10]), (1, list(range(11))),
                                         (3, [0, 3, 4, 7, 10]), (5, [0, 4, 9, 10])])
def test_bj_blocks_by_hand(orc, max_bs, want):
    """Rows 0-2 share one column list, row 3 has its own, rows 4-9 share a
    third: supervariables of 3, 1 and 6 rows.  The expected boundaries are
    worked out by hand from the two steps (cut at max_bs, merge greedily)."""
    rows = [([0, 1, 2], [4.0, 1.0, 1.0])] * 3 + [([3], [2.0])] + [(list(range(4, 10)), [1.0] * 6)] * 6
    A = _csr_rows(10, rows)
    assert orc.bj_blocks(A, max_bs).tolist() == want


def test_bj_blocks_distinct_rows_and_empty_runs(orc):
    """Every row of the 1-D Laplacian has its own column list: blocks of
    max_bs rows and a short tail.  A run of empty rows is one supervariable
    (identical, empty lists)."""
    A = _laplace1d(70)
    assert orc.bj_blocks(A, 8).tolist() == list(range(0, 70, 8)) + [70]
    assert orc.bj_blocks(A, 32).tolist() == [0, 32, 64, 70]
    E = _csr_rows(9, [([0], [1.0]), ([1], [1.0])] + [([], [])] * 5 + [([7], [1.0]), ([8], [1.0])])
    # pieces 1, 1 | 4 empty rows (the run cut at 4) | the fifth empty row, 1, 1 merged
    assert orc.bj_blocks(E, 4).tolist() == [0, 2, 6, 9]
    assert orc.bj_blocks(_csr_rows(0, []), 8).tolist() == [0]
    with pytest.raises(ValueError):
        orc.bj_blocks(A, 33)


@pytest.mark.parametrize("max_bs", [8, 5, 32])
def test_bj_invert_tridiagonal_closed_form(orc, max_bs):
    """The diagonal blocks of the 1-D Laplacian are tridiag(-1, 2, -1) of
    order s, whose inverse is min(i, j) (s + 1 - max(i, j)) / (s + 1) with
    1-based i, j."""
    n = 70
    A = _laplace1d(n)
    bp = orc.bj_blocks(A, max_bs)
    st, inv = orc.bj_invert(A, bp, max_bs)
    assert st == orc.OK
    for o, e in zip(bp[:-1], bp[1:]):
        s = e - o
        for i in range(s):
            for j in range(s):
                want = min(i + 1, j + 1) * (s + 1 - max(i + 1, j + 1)) / (s + 1)
                assert abs(inv[o * max_bs + j * s + i] - want) <= 1e-13 * s, (o, s, i, j)


def test_bj_invert_layout_lower_triangular(orc):
    """A = I + a S (S the subdiagonal): every diagonal block of 4 rows is
    unit lower bidiagonal, with inverse (-a)^(i-j) for i >= j and 0 above
    the diagonal; the stored layout (column j, row i at j * s + i) puts the
    nonzeros below the diagonal, so a transposed store fails."""
    a = 0.75
    n = 12
    rows = [([0], [1.0])] + [([i - 1, i], [a, 1.0]) for i in range(1, n)]
    A = _csr_rows(n, rows)
    bp = orc.bj_blocks(A, 4)
    assert bp.tolist() == [0, 4, 8, 12]
    st, inv = orc.bj_invert(A, bp, 4)
    assert st == orc.OK
    for o in (0, 4, 8):
        for i in range(4):
            for j in range(4):
                want = (-a) ** (i - j) if i >= j else 0.0
                assert abs(inv[o * 4 + j * 4 + i] - want) <= 1e-15


@pytest.mark.parametrize("max_bs", [3, 8, 32])
def test_bj_invert_and_apply_match_numpy(orc, max_bs):
    """Non-symmetric diagonally dominant matrix: each stored inverse equals
    numpy's inverse of the block the test extracts from the dense matrix,
    and z = M^-1 r equals numpy's block solves."""
    A = syn.random_csr(300, 300, 12, seed=31)
    n = 300
    D = dense(A)
    D[np.arange(n), np.arange(n)] += 20.0
    keep = D != 0
    r_i, c_i = np.nonzero(keep)
    B = dict(n_rows=n, n_cols=n, row_ptr=np.concatenate([[0], np.cumsum(keep.sum(1))]).astype(np.int32),
             col_idx=c_i.astype(np.int32), val=D[r_i, c_i])
    bp = orc.bj_blocks(B, max_bs)
    st, inv = orc.bj_invert(B, bp, max_bs)
    assert st == orc.OK
    r = syn.vector(n, 32)
    z = orc.bj_apply(bp, max_bs, inv, r)
    for o, e in zip(bp[:-1], bp[1:]):
        s = e - o
        Bk = D[o:e, o:e]
        got = inv[o * max_bs:o * max_bs + s * s].reshape(s, s).T  # column-major
        assert np.allclose(got, np.linalg.inv(Bk), rtol=0, atol=1e-14)
        assert np.allclose(z[o:e], np.linalg.solve(Bk, r[o:e]), rtol=0, atol=1e-13)


def test_bj_singular_block_is_breakdown(orc):
    A = _laplace1d(16)
    Z = dict(A)
    Z["val"] = A["val"].copy()
    Z["val"][A["row_ptr"][5]:A["row_ptr"][6]] = 0.0  # row 5 zero: its block is singular
    st, _ = orc.bj_invert(Z, orc.bj_blocks(Z, 4), 4)
    assert st == orc.BREAKDOWN
    b = syn.vector(16, 3)
    x, st, it, res = orc.pcg_block_jacobi(Z, b, 4)
    assert st == orc.BREAKDOWN and it == 0


def _spd_block_diagonal(n, b, seed):
    """Block-diagonal SPD matrix: each dense b x b block R R^T + b I."""
    A = syn.block_diagonal(n, b, seed=seed)
    D = dense(A)
    S = np.zeros_like(D)
    for o in range(0, n, b):
        R = D[o:o + b, o:o + b]
        S[o:o + b, o:o + b] = R @ R.T + b * np.eye(b)
    r_i, c_i = np.nonzero(S)
    return dict(n_rows=n, n_cols=n, row_ptr=np.concatenate([[0], np.cumsum((S != 0).sum(1))]).astype(np.int32),
                col_idx=c_i.astype(np.int32), val=S[r_i, c_i])


def test_pcg_block_jacobi_exact_preconditioner_one_step(orc):
    """Rows of one dense 8 x 8 block share a column list, so with
    max_bs = 8 the blocks are A's own blocks, M = A, and one step gives
    alpha = 1 and the exact solution."""
    A = _spd_block_diagonal(64, 8, seed=33)
    assert orc.bj_blocks(A, 8).tolist() == list(range(0, 65, 8))
    xt = syn.vector(64, 34)
    b = dense(A) @ xt
    x, st, it, res = orc.pcg_block_jacobi(A, b, 8, tol=1e-13)
    assert st == orc.OK and it == 1
    assert np.linalg.norm(x - xt) <= 1e-13 * np.linalg.norm(xt)


def test_pcg_block_jacobi_size_one_is_jacobi(orc):
    """Blocks of one row: M = diag(A), the iterates of Jacobi PCG."""
    A = _scaled(syn.laplace2d(24), 10.0 ** (2.0 * syn.uniform01(35, 1, np.arange(576, dtype=np.uint64))))
    b = orc.spmv_csr(A, syn.vector(576, 36))
    for k in (1, 4, 20):
        xa, _, _, _ = orc.pcg_jacobi(A, b, maxit=k)
        xb, _, ib, _ = orc.pcg_block_jacobi(A, b, 1, maxit=k)
        assert ib == k and np.linalg.norm(xa - xb) <= 1e-11 * np.linalg.norm(xa)
    _, s0, i0, _ = orc.pcg_jacobi(A, b, tol=1e-10)
    _, s1, i1, r1 = orc.pcg_block_jacobi(A, b, 1, tol=1e-10)
    assert s0 == s1 == orc.OK and abs(i0 - i1) <= 1 and r1 <= 1e-10


def test_pcg_block_jacobi_diffusion(orc):
    """7-point diffusion: larger blocks (consecutive rows along x) take
    fewer steps than point Jacobi, and the solve reaches the manufactured
    solution with a confirmed true residual."""
    A = syn.diffusion7(12, 1.0, seed=6)
    n = A["n_rows"]
    xt = syn.vector(n, 37)
    b = orc.spmv_csr(A, xt)
    _, s0, i0, _ = orc.pcg_jacobi(A, b, tol=1e-10)
    x, st, it, res = orc.pcg_block_jacobi(A, b, 12, tol=1e-10)
    assert s0 == st == orc.OK and res <= 1e-10 and it < i0
    assert orc.true_rel_residual(A, b, x) <= 1e-10
    assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)
    xd = np.linalg.solve(dense(A), b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)


def test_pcg_block_jacobi_special_cases(orc):
    A = _laplace1d(40)
    x, st, it, res = orc.pcg_block_jacobi(A, np.zeros(40), 8, x0=np.ones(40))
    assert st == orc.OK and it == 0 and np.all(x == 0)
    b = orc.spmv_csr(A, syn.vector(40, 2))
    x, st, it, res = orc.pcg_block_jacobi(A, b, 8, maxit=3)
    assert st == orc.NOT_CONVERGED and it == 3
    # one block holding the whole matrix: M = A, one step
    x, st, it, res = orc.pcg_block_jacobi(_laplace1d(20), orc.spmv_csr(_laplace1d(20), np.ones(20)), 32)
    assert st == orc.OK and it == 1 and np.allclose(x, 1.0, rtol=0, atol=1e-13)


def test_bicgstab_scaled_identity_one_step(orc):
    """A = c I: v = c p, alpha = 1/c, s = 0 after the first half step, so
    x = b / c exactly (a closed form of one step)."""
    n = 50
    A = _diag_spd(np.full(n, 2.5))
    b = syn.vector(n, 31)
    x, st, it, res = orc.bicgstab(A, b, tol=1e-14)
    assert st == orc.OK and it == 1
    assert np.allclose(x, b / 2.5, rtol=1e-15, atol=0)


def test_bicgstab_finite_termination(orc):
    """BiCGSTAB's residual is psi_k(A) phi_k(A) r0 with phi_k the BiCG
    polynomial, which annihilates r0 once k reaches the degree of the
    minimal polynomial: a diagonalizable nonsymmetric matrix with three
    distinct eigenvalues (upper-triangular 2x2 blocks with eigenvalue pairs
    from {1, 2, 3}) is solved in at most three steps."""
    blocks = [((1.0, 0.7), (0.0, 2.0)), ((2.0, 0.3), (0.0, 3.0)), ((3.0, -0.5), (0.0, 1.0))]
    nb = 30
    rp, ci, va = [0], [], []
    for k in range(nb):
        (a, b_), (_, c) = blocks[k % 3]
        r0 = 2 * k
        ci += [r0, r0 + 1]; va += [a, b_]; rp.append(len(ci))
        ci += [r0 + 1]; va += [c]; rp.append(len(ci))
    A = dict(n_rows=2 * nb, n_cols=2 * nb, row_ptr=np.array(rp, np.int32), col_idx=np.array(ci, np.int32),
             val=np.array(va))
    b = syn.vector(2 * nb, 33)
    x, st, it, res = orc.bicgstab(A, b, tol=1e-12)
    assert st == orc.OK and it <= 3, (st, it, res)
    assert np.allclose(dense(A) @ x, b, rtol=0, atol=1e-11)


def test_bicgstab_matches_dense_solve(orc):
    """Small nonsymmetric systems (random sparse, made diagonally dominant)
    against numpy's dense LU solve."""
    for seed in (41, 42, 43):
        A = syn.random_csr(120, 120, 6, seed=seed)
        n = 120
        rows = np.repeat(np.arange(n), np.diff(A["row_ptr"]))
        D = dense(A)
        D = D + np.diag(1.0 + np.abs(D).sum(axis=1))
        # write the dominant diagonal back into a CSR with every diagonal stored
        Dm = np.where(np.abs(D) > 0, D, 0.0)
        rp = np.concatenate([[0], np.cumsum((Dm != 0).sum(axis=1))]).astype(np.int32)
        ci = np.nonzero(Dm)[1].astype(np.int32)
        B = dict(n_rows=n, n_cols=n, row_ptr=rp, col_idx=ci, val=Dm[Dm != 0])
        b = syn.vector(n, seed)
        x, st, it, res = orc.bicgstab(B, b, tol=1e-13)
        assert st == orc.OK and res <= 1e-13
        assert np.allclose(x, np.linalg.solve(Dm, b), rtol=1e-10, atol=1e-12)


def test_bicgstab_convection_diffusion(orc):
    """Nonsymmetric convection-diffusion: BiCGSTAB reaches the manufactured
    solution; its recursive residual agrees with b - A x at the end."""
    A = syn.convdiff2d(48, 0.8)
    n = A["n_rows"]
    D = dense(A)
    assert not np.allclose(D, D.T)
    xt = syn.vector(n, 32)
    b = orc.spmv_csr(A, xt)
    x, st, it, res = orc.bicgstab(A, b, tol=1e-10)
    assert st == orc.OK and res <= 1e-10
    cond = np.linalg.cond(D)
    assert np.linalg.norm(x - xt) <= cond * 1e-10 * np.linalg.norm(xt)
    assert it < n // 4


def test_bicgstab_special_cases(orc):
    A = syn.convdiff2d(8, 0.5)
    n = A["n_rows"]
    x, st, it, res = orc.bicgstab(A, np.zeros(n), x0=np.ones(n))
    assert st == orc.OK and it == 0 and np.all(x == 0)
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x, st, it, res = orc.bicgstab(A, b, maxit=2)
    assert st == orc.NOT_CONVERGED and it == 2
    x, st, it, res = orc.bicgstab(A, b, x0=syn.vector(n, 2))
    assert st == orc.OK and it == 0
    # rho' = r^.r = 0 cannot happen for r != 0; A = 0 gives r^.v = 0: breakdown
    Z = dict(A)
    Z["val"] = np.zeros_like(A["val"])
    x, st, it, res = orc.bicgstab(Z, b)
    assert st == orc.BREAKDOWN


def test_spmm_columns_are_spmvs_and_identity_gives_dense(orc):
    """SpMM pins: with X = the identity the block is the dense matrix
    (brute force); every column equals the SpMV of that column (integer
    values: exact); alpha/beta as in SpMV."""
    A = syn.random_csr(37, 23, 5, seed=51, empty_frac=0.2)
    D = dense(A)
    Y = orc.spmm_csr(A, np.eye(23))
    assert np.array_equal(Y, D)
    rng = np.random.default_rng(52)
    Ai = dict(A)
    Ai["val"] = rng.integers(-5, 6, size=len(A["val"])).astype(np.float64)
    X = rng.integers(-5, 6, size=(23, 6)).astype(np.float64)
    Y0 = rng.integers(-5, 6, size=(37, 6)).astype(np.float64)
    Y = orc.spmm_csr(Ai, X, 2.0, -1.0, Y0)
    assert np.array_equal(Y, 2.0 * dense(Ai) @ X - Y0)
    for c in range(6):
        assert np.array_equal(Y[:, c], orc.spmv_csr(Ai, X[:, c], 2.0, -1.0, Y0[:, c]))


def test_gmres_finite_termination(orc):
    """m distinct eigenvalues (the 3-eigenvalue nonsymmetric block matrix of
    the BiCGSTAB pin): GMRES without restart solves in at most 3 steps."""
    blocks = [((1.0, 0.7), (0.0, 2.0)), ((2.0, 0.3), (0.0, 3.0)), ((3.0, -0.5), (0.0, 1.0))]
    nb = 30
    rp, ci, va = [0], [], []
    for k in range(nb):
        (a, b_), (_, c) = blocks[k % 3]
        r0 = 2 * k
        ci += [r0, r0 + 1]; va += [a, b_]; rp.append(len(ci))
        ci += [r0 + 1]; va += [c]; rp.append(len(ci))
    A = dict(n_rows=2 * nb, n_cols=2 * nb, row_ptr=np.array(rp, np.int32), col_idx=np.array(ci, np.int32),
             val=np.array(va))
    b = syn.vector(2 * nb, 34)
    x, st, it, res = orc.gmres(A, b, tol=1e-12, restart=50)
    assert st == orc.OK and it <= 3, (st, it)


def test_gmres_minimal_residual_below_cg(orc):
    """GMRES minimises ||b - A x|| over the Krylov space that CG's iterate
    also lies in: after k steps (no restart, x0 = 0) its true residual is no
    larger than CG's on an SPD matrix."""
    A = syn.diffusion7(8, 1.0, seed=5)
    n = A["n_rows"]
    b = syn.vector(n, 35)
    for k in (1, 2, 5, 10, 20):
        _, _, _, rg = orc.gmres(A, b, tol=1e-300, restart=100, maxit=k)
        _, _, _, rc = orc.cg(A, b, tol=1e-300, maxit=k)
        assert rg <= rc * (1 + 1e-10), (k, rg, rc)


def test_gmres_matches_dense_and_restarts(orc):
    A = syn.convdiff2d(24, 0.8)
    n = A["n_rows"]
    xt = syn.vector(n, 36)
    b = orc.spmv_csr(A, xt)
    x, st, it, res = orc.gmres(A, b, tol=1e-11, restart=40)
    assert st == orc.OK and res <= 1e-11
    assert np.allclose(x, np.linalg.solve(dense(A), b), rtol=1e-8, atol=1e-10)
    # a shorter restart needs at least as many steps and still converges
    x2, st2, it2, res2 = orc.gmres(A, b, tol=1e-11, restart=10)
    assert st2 == orc.OK and it2 >= it


def test_gmres_special_cases(orc):
    A = syn.convdiff2d(8, 0.5)
    n = A["n_rows"]
    x, st, it, res = orc.gmres(A, np.zeros(n), x0=np.ones(n))
    assert st == orc.OK and it == 0 and np.all(x == 0)
    b = orc.spmv_csr(A, syn.vector(n, 2))
    x, st, it, res = orc.gmres(A, b, maxit=3)
    assert st == orc.NOT_CONVERGED and it == 3
    x, st, it, res = orc.gmres(A, b, x0=syn.vector(n, 2))
    assert st == orc.OK and it == 0


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_cg_jacobi_inner(orc, prec):
    """Jacobi-preconditioned inner solve: it reaches the FP64 residual with
    several times fewer inner steps than the unpreconditioned inner solve
    (FP32 storage: diffusion operator rescaled over three decades; BF16
    storage, whose 8-bit significand cannot hold that scaled operator: the
    variable-coefficient diffusion operator itself); a constant diagonal
    (Laplacian) leaves the inner iterates unchanged."""
    A0 = syn.diffusion7(12, 1.0, seed=6)
    n = A0["n_rows"]
    if prec == "fp32":
        s = 10.0 ** (3.0 * syn.uniform01(27, 1, np.arange(n, dtype=np.uint64)))
        A, factor = _scaled(A0, s), 3
    else:
        A, factor = A0, 1
    b = orc.spmv_csr(A, syn.vector(n, 28))
    xj, stj, oj, ij, rj = orc.cg_mixed(A, b, prec, tol=1e-10, inner_tol=1e-2, precond="jacobi")
    xn, stn, on, in_, rn = orc.cg_mixed(A, b, prec, tol=1e-10, inner_tol=1e-2, maxit_outer=400)
    assert stj == orc.OK and rj <= 1e-10
    assert ij * factor < in_, (ij, in_)
    L = syn.laplace2d(20)
    bl = orc.spmv_csr(L, syn.vector(400, 29))
    r1 = orc.cg_mixed(L, bl, prec, tol=1e-10, inner_tol=1e-3)
    r2 = orc.cg_mixed(L, bl, prec, tol=1e-10, inner_tol=1e-3, precond="jacobi")
    assert r1[2] == r2[2] and abs(r1[3] - r2[3]) <= 2 and r2[4] <= 1e-10


def _batch_dense(B, k):
    r0, r1 = int(B["row_off"][k]), int(B["row_off"][k + 1])
    D = np.zeros((r1 - r0, r1 - r0))
    for i in range(r0, r1):
        for e in range(B["row_ptr"][i], B["row_ptr"][i + 1]):
            D[i - r0, B["col_idx"][e]] += B["val"][e]
    return D, r0, r1


def test_batched_cg(orc):
    """Every system's solution against numpy's dense solve (the systems are
    strictly diagonally dominant, so cond(A) is small and a relative residual
    of 1e-10 bounds the error near 1e-10 too), and the reported residual
    recomputed from x."""
    B = syn.batched_spd(12, seed=8)
    x, st, it, res = orc.cg_batched(B, B["rhs"], tol=1e-10)
    assert np.all(st == 0) and np.all(res <= 1e-10)
    assert np.all(it > 0)
    for k in range(12):
        D, r0, r1 = _batch_dense(B, k)
        b = B["rhs"][r0:r1]
        xs = np.linalg.solve(D, b)
        assert np.linalg.norm(x[r0:r1] - xs) <= 1e-8 * np.linalg.norm(xs)
        rr = np.linalg.norm(b - D @ x[r0:r1]) / np.linalg.norm(b)
        assert abs(rr - res[k]) <= 1e-13


def test_batched_cg_finite_termination_and_special_systems(orc):
    """CG ends after at most m steps on a matrix with m distinct eigenvalues
    (diagonal systems with 1, 2 and 3 distinct entries), takes one step on a
    1x1 system, and returns x = 0 after no step when b = 0."""
    diags = [np.full(7, 3.0), np.array([2.0, 5.0, 2.0, 5.0, 5.0]), np.array([1.0, 4.0, 9.0, 1.0, 4.0, 9.0]),
             np.array([2.5]), np.array([3.0, 1.0, 2.0])]
    ro = np.concatenate([[0], np.cumsum([len(d) for d in diags])]).astype(np.int64)
    rp = np.arange(ro[-1] + 1, dtype=np.int32)
    ci = np.concatenate([np.arange(len(d)) for d in diags]).astype(np.int32)
    B = dict(row_off=ro, row_ptr=rp, col_idx=ci, val=np.concatenate(diags), sizes=np.diff(ro))
    b = syn.vector(int(ro[-1]), 17)
    b[ro[4]:ro[5]] = 0.0  # last system: b = 0
    x, st, it, res = orc.cg_batched(B, b, tol=1e-12)
    assert np.all(st == 0)
    assert list(it) == [1, 2, 3, 1, 0]
    for k in range(4):
        r0, r1 = ro[k], ro[k + 1]
        assert np.allclose(x[r0:r1], b[r0:r1] / diags[k], rtol=1e-12, atol=0)
    assert np.all(x[ro[4]:ro[5]] == 0.0) and res[4] == 0.0


# --------------------------------------------------------- mixed precision

def _bf16_neighbours(v):
    """All bfloat16 values adjacent to v, by enumeration of float32 bit patterns."""
    f = np.float32(v)
    bits = int(np.array(f, dtype=np.float32).view(np.uint32)) & 0xFFFF0000
    cands = []
    for dlt in (-2, -1, 0, 1, 2):
        bb = (bits + dlt * 0x10000) & 0xFFFFFFFF
        cands.append(float(np.array(bb, dtype=np.uint32).view(np.float32)))
    return sorted(set(cands))


def test_round_bf16_by_enumeration(orc):
    rng = np.random.default_rng(7)
    vals = list(rng.standard_normal(400) * 10.0 ** rng.integers(-5, 5, 400))
    vals += [1.0, 1.00390625, 1.001953125, 1.005859375, -1.001953125, 3.0 + 2 ** -7, 255.5]
    for v in vals:
        c = _bf16_neighbours(v)
        dist = [abs(Fraction(u) - Fraction(v)) for u in c]
        best = min(dist)
        winners = [u for u, d in zip(c, dist) if d == best]
        if len(winners) > 1:  # tie: the even significand (low bit of the bf16 pattern clear)
            winners = [u for u in winners
                       if (int(np.array(np.float32(u)).view(np.uint32)) >> 16) % 2 == 0]
        assert orc.round_bf16(v) == winners[0], v
        up = min(u for u in c if u >= v)
        assert orc.round_bf16(v, up=True) == up, v


def test_round_fp32_matches_ieee_cast(orc):
    rng = np.random.default_rng(8)
    for v in rng.standard_normal(1000) * 10.0 ** rng.integers(-20, 20, 1000):
        assert orc.round_fp32(v) == float(np.float32(v))
        u = orc.round_fp32(v, up=True)
        assert u >= v and float(np.nextafter(np.float32(u), np.float32(-np.inf))) < v


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_round_matrix_preserves_row_sums(orc, prec):
    """Off-diagonals are the nearest low-precision values; the diagonal is
    the nearest value to the row-sum-preserving target, so every row sum of
    the copy is within half an ulp of the diagonal of the original's."""
    A = syn.diffusion7(10, 1.0, seed=6)
    lo = orc.round_matrix(A, prec)
    rp, ci = A["row_ptr"], A["col_idx"]
    bits = 8 if prec == "bf16" else 24
    for i in range(A["n_rows"]):
        ks = range(rp[i], rp[i + 1])
        off = [k for k in ks if ci[k] != i]
        kd = [k for k in ks if ci[k] == i][0]
        for k in off:
            r = orc.round_bf16(A["val"][k]) if prec == "bf16" else float(np.float32(A["val"][k]))
            assert lo[k] == r
        target = Fraction(A["val"][kd]) + sum(Fraction(abs(lo[k])) - Fraction(abs(A["val"][k])) for k in off)
        half_ulp = Fraction(2) ** (math.frexp(float(target))[1] - bits - 1)
        # the target itself is formed in FP64: allow a few FP64 ulps on top
        slack = Fraction(8) * Fraction(2) ** -52 * abs(target)
        assert abs(Fraction(lo[kd]) - target) <= half_ulp + slack
        row_sum = sum(Fraction(A["val"][k]) for k in ks)
        row_sum_lo = sum(Fraction(lo[k]) for k in ks)
        assert abs(row_sum_lo - row_sum) <= half_ulp + slack


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_cg_reaches_fp64_accuracy(orc, prec):
    A = syn.diffusion7(16, 1.0, seed=6)
    n = A["n_rows"]
    xt = syn.vector(n, 6)
    b = orc.spmv_csr(A, xt)
    x64, st, it, res = orc.cg(A, b, tol=1e-10)
    x, st, outer, inner, res = orc.cg_mixed(A, b, prec, tol=1e-10, inner_tol=1e-3)
    assert st == orc.OK and res <= 1e-10
    assert 1 <= outer <= 30
    assert np.linalg.norm(x - x64) <= 1e-8 * np.linalg.norm(x64)


# ---------------------------------------------------------------- features

def test_features_brute_force(orc):
    for A in small_mats() + [syn.laplace2d(16), syn.banded(500, 64, 16, seed=3)]:
        n = A["n_rows"]
        L = [int(A["row_ptr"][i + 1] - A["row_ptr"][i]) for i in range(n)]
        nnz = sum(L)
        mean = nnz / n
        ent = [(i, int(A["col_idx"][k])) for i in range(n) for k in range(A["row_ptr"][i], A["row_ptr"][i + 1])]
        slots = sum(32 * max(L[s:s + 32]) for s in range(0, n, 32))
        exp = [math.log10(n), math.log10(max(nnz, 1)), mean,
               math.sqrt(sum((l - mean) ** 2 for l in L) / n), max(L), min(L),
               max(L) / mean if mean else 0.0, sum(l == 0 for l in L) / n,
               max((abs(i - j) for i, j in ent), default=0) / n,
               (sum(abs(i - j) for i, j in ent) / nnz / n) if nnz else 0.0,
               sum(1 for i, j in ent if i == j) / n, slots / nnz if nnz else 0.0]
        f = orc.features(A)
        assert np.allclose(f, exp, rtol=1e-12, atol=0), (f, exp)


def test_features_closed_form_laplacian_16():
    """5-point Laplacian on a 16 x 16 grid, every statistic worked out by hand:
    4 corner rows of 3 entries, 56 edge rows of 4, 196 interior rows of 5
    (nnz 1216); 480 entries with |i-j| = 1, 480 with |i-j| = 16, 256 on the
    diagonal; every 32-row SELL-P slice holds an interior row (width 5).
    Catches a sample (n-1) instead of population std, |i-j| averaged over
    rows instead of entries, and a SELL-P width taken from the mean."""
    f = orc_features_of(syn.laplace2d(16))
    exp = [math.log10(256), math.log10(1216), 4.75, math.sqrt(56 / 256), 5, 3, 5 / 4.75, 0.0,
           16 / 256, 8160 / 1216 / 256, 1.0, 1280 / 1216]
    assert np.allclose(f, exp, rtol=1e-13, atol=0), (f, exp)


def test_features_closed_form_block_diagonal():
    """Five dense 8 x 8 blocks (n = 40): rows of 8, bandwidth 7, sum of
    |i-j| over one block 2 (7 + 12 + 15 + 16 + 15 + 12 + 7) = 168, i.e. 2.625
    per entry; the last SELL-P slice (8 rows) still counts 32 rows of
    width 8, so the slots are 512 for 320 entries."""
    f = orc_features_of(syn.block_diagonal(40, 8, seed=5))
    exp = [math.log10(40), math.log10(320), 8.0, 0.0, 8, 8, 1.0, 0.0, 7 / 40, 2.625 / 40, 1.0, 512 / 320]
    assert np.allclose(f, exp, rtol=1e-13, atol=1e-300), (f, exp)


def test_features_closed_form_half_empty_diagonal():
    """Diagonal entries in the even rows of a 64 x 64 matrix, odd rows empty:
    mean 1/2, population std 1/2, min 0, max/mean 2, half the rows empty and
    half holding their diagonal, two SELL-P slices of width 1 (64 slots for
    32 entries)."""
    n = 64
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(np.arange(n) % 2 == 0)
    A = dict(n_rows=n, n_cols=n, row_ptr=rp, col_idx=np.arange(0, n, 2, dtype=np.int32), val=np.ones(n // 2))
    f = orc_features_of(A)
    exp = [math.log10(64), math.log10(32), 0.5, 0.5, 1, 0, 2.0, 0.5, 0.0, 0.0, 0.5, 2.0]
    assert np.allclose(f, exp, rtol=1e-13, atol=1e-300), (f, exp)


def orc_features_of(A):
    import oracle
    oracle.build()
    return oracle.features(A)


# ---------------------------------------------------------------------- MLP

def test_mlp_gradient_central_differences():
    from oracle import mlp
    rng = np.random.default_rng(1)
    C = 5
    P = {k: rng.standard_normal(s) * 0.3 for k, s in mlp.shapes(12, 64, C).items()}
    X = rng.standard_normal((16, 12))
    Y = rng.standard_normal((16, C))
    M = (rng.random((16, C)) > 0.2).astype(float)
    L, g = mlp.loss_and_grad(P, X, Y, M)
    h = 1e-6
    for k in mlp.NAMES:
        flat = P[k].reshape(-1)
        for t in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[t]
            flat[t] = old + h
            lp = mlp.loss(P, X, Y, M)
            flat[t] = old - h
            lm = mlp.loss(P, X, Y, M)
            flat[t] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[t]) <= 1e-6 * max(1.0, abs(fd)), (k, t)


def test_adam_first_step_moves_by_lr():
    """At t = 1 Adam moves every parameter by lr * sign(g) (up to eps)."""
    from oracle import mlp
    P = {k: np.zeros(s) for k, s in mlp.shapes(12, 64, 3).items()}
    g = {k: np.full(s, 0.5) for k, s in mlp.shapes(12, 64, 3).items()}
    g["b3"][:] = -2.0
    P = mlp.adam_step(P, g, {}, 1, lr=0.01)
    assert np.allclose(P["W1"], -0.01, rtol=1e-6) and np.allclose(P["b3"], 0.01, rtol=1e-6)


def test_mlp_forward_hand_computed():
    """A sparse network whose output is worked out by hand: h1 = relu(W1 x + b1)
    = (2, relu(-3) = 0, 0.5); h2 = relu(W2 h1 + b2) = (2 + 10 * 0, 4 * 0.5,
    relu(-2) = 0, relu(-1) = 0); out = W3 h2 + b3 = (0.5 * 2 + 0.25 * 2 + 0.1,
    7 * 0 - 0.2).  A dropped ReLU, a dropped bias or a transposed W2/W3 each
    changes the result."""
    from oracle import mlp
    P = {k: np.zeros(s) for k, s in mlp.shapes(12, 64, 2).items()}
    P["W1"][0, 0], P["W1"][1, 1], P["b1"][2] = 1.0, -1.0, 0.5
    P["W2"][0, 0], P["W2"][0, 1], P["W2"][1, 2], P["W2"][2, 0], P["b2"][3] = 1.0, 10.0, 4.0, -1.0, -1.0
    P["W3"][0, 0], P["W3"][0, 1], P["W3"][1, 2], P["b3"][:] = 0.5, 0.25, 7.0, (0.1, -0.2)
    X = np.zeros((2, 12))
    X[0, :2] = (2.0, 3.0)
    X[1, :2] = (-1.0, 0.0)  # second sample: h1 = (0, 0, 0.5), h2 = (0, 2, 0, 0)
    out, _ = mlp.forward(P, X)
    assert np.allclose(out, [[1.6, -0.2], [0.25 * 2 + 0.1, -0.2]], rtol=0, atol=1e-15), out
    # masked MSE of that output: only (0, 0) and (1, 1) count
    Y = np.array([[1.0, 5.0], [0.0, 0.3]])
    M = np.array([[1.0, 0.0], [0.0, 1.0]])
    assert abs(mlp.loss(P, X, Y, M) - (0.6 ** 2 + 0.5 ** 2) / 2) <= 1e-15


def test_adam_bias_correction_after_three_steps():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2 at every step, so each of steps 1, 2, 3 moves a parameter by
    lr * sign(g) (up to eps): after three steps it sits at -3 lr sign(g).
    Without the 1 - beta^t corrections the second step would move by
    lr * 0.19 / sqrt(0.001999) = 4.25 lr."""
    from oracle import mlp
    sh = mlp.shapes(12, 64, 3)
    P = {k: np.zeros(s) for k, s in sh.items()}
    g = {k: np.full(s, 0.5) for k, s in sh.items()}
    g["b3"][:] = -2.0
    st = {}
    for t in (1, 2, 3):
        P = mlp.adam_step(P, g, st, t, lr=0.01)
        assert np.allclose(P["W1"], -0.01 * t, rtol=1e-6) and np.allclose(P["b3"], 0.01 * t, rtol=1e-6), t


def test_adam_two_steps_worked_example():
    """Gradients 1 then -2 with the default betas (0.9, 0.999), worked out by
    hand: m1 = 0.1, v1 = 0.001 -> step 1 = lr; m2 = 0.09 - 0.2 = -0.11,
    v2 = 0.000999 + 0.004 = 0.004999, m2^ = -0.11 / 0.19, v2^ = 0.004999 /
    0.001999, step 2 = lr m2^ / sqrt(v2^) = -0.366100... lr."""
    from oracle import mlp
    sh = {k: (1,) for k in mlp.NAMES}
    P = {k: np.zeros(1) for k in mlp.NAMES}
    st = {}
    P = mlp.adam_step(P, {k: np.ones(1) for k in sh}, st, 1, lr=1.0, eps=0.0)
    assert abs(P["W1"][0] + 1.0) <= 1e-12
    P = mlp.adam_step(P, {k: np.full(1, -2.0) for k in sh}, st, 2, lr=1.0, eps=0.0)
    step2 = (-0.11 / 0.19) / math.sqrt(0.004999 / 0.001999)
    assert abs(step2 + 0.3661) < 1e-4
    assert abs(P["W1"][0] - (-1.0 - step2)) <= 1e-12, P["W1"][0]


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_all_cores_row_loop_equals_the_oracle(orc, threads):
    """The OpenMP row loop of the CPU baseline computes each row exactly as
    the sequential oracle does: bit-identical results for any thread count."""
    for A in small_mats() + [syn.powerlaw(3000, 12.0, 1.5, 900, seed=42)]:
        x = syn.vector(A["n_cols"], 5)
        y0 = syn.vector(A["n_rows"], 6)
        a = orc.spmv_csr(A, x, 1.5, -0.5, y0)
        b = orc.spmv_csr_omp(A, x, threads, 1.5, -0.5, y0)
        assert np.array_equal(a, b)

def _indefinite_bf16_case(orc):
    """48 x 48 SPD matrix (eigenvalues 1e-6 and 1..2, seeded orthogonal basis)
    whose BF16 copy (rounding the diagonal to nearest) has an eigenvalue of
    -4e-4; b is that eigenvector, so the inner CG on A_lo meets p.Ap < 0 at
    its first step."""
    n = 48
    U = syn.uniform_pm1(10, 1, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    Q, _ = np.linalg.qr(U)
    lam = np.linspace(1.0, 2.0, n)
    lam[0] = 1e-6
    D = (Q * lam) @ Q.T
    D = 0.5 * (D + D.T)
    r, c = np.nonzero(D)
    A = dict(n_rows=n, n_cols=n, row_ptr=np.concatenate([[0], np.cumsum((D != 0).sum(1))]).astype(np.int32),
             col_idx=c.astype(np.int32), val=D[r, c])
    Dl = np.zeros((n, n))
    Dl[r, c] = orc.round_matrix(A, "bf16")
    ev, V = np.linalg.eigh(0.5 * (Dl + Dl.T))
    return A, V[:, 0], ev[0], np.linalg.eigvalsh(D)[0]


def test_mixed_cg_inner_breakdown_on_indefinite_copy(orc):
    """Rounding the diagonal to nearest can leave A_lo indefinite though A is
    SPD.  The inner CG then stops at its breakdown (p.Ap <= 0) and the outer
    loop keeps its FP64 residual: no NaN, no progress along that direction,
    NOT_CONVERGED after maxit_outer corrections of one inner step each."""
    A, b, lo_min, a_min = _indefinite_bf16_case(orc)
    assert a_min > 0 and lo_min < -1e-4
    x, st, o, i, res = orc.cg_mixed(A, b, prec="bf16", tol=1e-10, maxit_outer=5, inner_tol=1e-1)
    assert st == orc.NOT_CONVERGED and o == 5 and i == 5
    assert np.all(np.isfinite(x)) and abs(res - 1.0) < 1e-12

