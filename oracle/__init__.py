"""Plain FP64 CPU oracle (test infrastructure only).

Only the tests, the package's smoke check and the benchmark's CPU-baseline
and reference legs (the oracle timed on the host cores) may import this
package.  The product path (the CUDA library and its
Python binding) never does, and the oracle shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C loops, compiled without fused
multiply-add) and in ``mlp.py`` (numpy, FP64).  This module only marshals
numpy arrays into those C routines.  Matrices are the CSR dicts of the
``synthetic`` module: ``n_rows, n_cols, row_ptr (int32), col_idx (int32),
val (float64)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")

OK, NOT_CONVERGED, BREAKDOWN = 0, 6, 7


OMP_LIB_PATH = os.path.join(HERE, "liboracle_omp.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (no FMA contraction), and
    the all-cores row loop oracle_omp.c into liboracle_omp.so (OpenMP)."""
    for src, out, extra in ((os.path.join(HERE, "oracle.c"), LIB_PATH, []),
                            (os.path.join(HERE, "oracle_omp.c"), OMP_LIB_PATH, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
            tmp = out + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", *extra,
                                   "-shared", "-o", tmp, src, "-lm"])
            os.replace(tmp, out)
    return LIB_PATH


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB_PATH)
        _declare(_lib)
    return _lib


_P = C.c_void_p
_I64 = C.c_int64
_D = C.c_double
_INT = C.c_int


def _declare(L):
    sig = {
        "orc_spmv_csr": (None, [_I64, _P, _P, _P, _P, _D, _D, _P]),
        "orc_spmv_csr_dot2": (None, [_I64, _P, _P, _P, _P, _D, _D, _P, _P, _P]),
        "orc_spmv_coo": (None, [_I64, _I64, _P, _P, _P, _P, _D, _D, _P]),
        "orc_spmv_ell": (None, [_I64, _I64, _I64, _P, _P, _P, _D, _D, _P]),
        "orc_spmv_sellp": (None, [_I64, _I64, _P, _P, _P, _P, _P, _D, _D, _P]),
        "orc_spmv_hybrid": (None, [_I64, _I64, _I64, _P, _P, _I64, _P, _P, _P, _P, _D, _D, _P]),
        "orc_csr_to_coo": (None, [_I64, _P, _P, _P, _P, _P, _P]),
        "orc_coo_to_csr": (None, [_I64, _I64, _P, _P, _P, _P, _P, _P]),
        "orc_max_row_len": (_I64, [_I64, _P]),
        "orc_ell_n_pad": (_I64, [_I64]),
        "orc_csr_to_ell": (None, [_I64, _I64, _I64, _P, _P, _P, _P, _P]),
        "orc_ell_to_csr": (None, [_I64, _I64, _I64, _P, _P, _P, _P, _P]),
        "orc_sellp_sizes": (_I64, [_I64, _P, _I64, _I64, _P, _P]),
        "orc_csr_to_sellp": (None, [_I64, _I64, _P, _P, _P, _P, _P, _P, _P]),
        "orc_sellp_to_csr": (None, [_I64, _I64, _P, _P, _P, _P, _P, _P, _P]),
        "orc_hybrid_width": (_I64, [_I64, _P, _I64]),
        "orc_hybrid_coo_nnz": (_I64, [_I64, _P, _I64]),
        "orc_csr_to_hybrid": (None, [_I64, _I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
        "orc_hybrid_to_csr": (None, [_I64, _I64, _I64, _P, _P, _I64, _P, _P, _P, _P, _P, _P]),
        "orc_dot": (_D, [_I64, _P, _P]),
        "orc_dot2": (_D, [_I64, _P, _P]),
        "orc_true_rel_residual": (_D, [_I64, _P, _P, _P, _P, _P]),
        "orc_cg": (_INT, [_I64, _P, _P, _P, _P, _P, _D, _INT, _P, _P]),
        "orc_cg_single_reduction": (_INT, [_I64, _P, _P, _P, _P, _P, _D, _INT, _P, _P]),
        "orc_pcg_jacobi": (_INT, [_I64, _P, _P, _P, _P, _P, _D, _INT, _P, _P]),
        "orc_bj_blocks": (_INT, [_I64, _P, _P, _INT, _P, _P]),
        "orc_bj_invert": (_INT, [_I64, _P, _P, _P, _INT, _P, _I64, _P]),
        "orc_bj_apply": (None, [_INT, _P, _I64, _P, _P, _P]),
        "orc_pcg_block_jacobi": (_INT, [_I64, _P, _P, _P, _INT, _P, _P, _D, _INT, _P, _P]),
        "orc_bicgstab": (_INT, [_I64, _P, _P, _P, _P, _P, _D, _INT, _P, _P]),
        "orc_spmm_csr": (None, [_I64, _P, _P, _P, _I64, _P, _I64, _D, _D, _P, _I64]),
        "orc_gmres": (_INT, [_I64, _P, _P, _P, _P, _P, _D, _INT, _INT, _P, _P]),
        "orc_cg_batched": (_INT, [_I64, _P, _P, _P, _P, _P, _P, _D, _INT, _P, _P, _P]),
        "orc_round_bf16": (_D, [_D, _INT]),
        "orc_round_fp32": (_D, [_D, _INT]),
        "orc_round_matrix": (None, [_I64, _P, _P, _P, _INT, _P]),
        "orc_cg_mixed": (_INT, [_I64, _P, _P, _P, _P, _P, _P, _D, _INT, _D, _INT, _P, _P, _P]),
        "orc_cg_mixed_precond": (_INT, [_I64, _P, _P, _P, _P, _P, _P, _D, _INT, _D, _INT, _INT, _P, _P, _P]),
        "orc_cholesky_solve": (_INT, [_I64, _P, _P, _P]),
        "orc_features": (None, [_I64, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a):
    return a.ctypes.data if a is not None and a.size else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _csr(A):
    return (int(A["n_rows"]), _c(A["row_ptr"], np.int32), _c(A["col_idx"], np.int32),
            _c(A["val"], np.float64))


# ------------------------------------------------------------------ SpMV

def spmv_csr(A, x, alpha=1.0, beta=0.0, y=None):
    """y = alpha A x + beta y (plain definition, row sums in column order)."""
    n, rp, ci, v = _csr(A)
    x = _c(x, np.float64)
    out = np.zeros(n) if y is None else np.array(y, dtype=np.float64, copy=True)
    lib().orc_spmv_csr(n, _p(rp), _p(ci), _p(v), _p(x), alpha, beta, _p(out))
    return out


_omp = None


def spmv_csr_omp(A, x, threads, alpha=1.0, beta=0.0, y=None):
    """spmv_csr with the row loop shared among `threads` host threads
    (OpenMP, static blocks of rows); bit-identical to spmv_csr."""
    global _omp
    if _omp is None:
        build()
        _omp = C.CDLL(OMP_LIB_PATH)
        _omp.orc_spmv_csr_omp.restype = None
        _omp.orc_spmv_csr_omp.argtypes = [_I64, _P, _P, _P, _P, _D, _D, _P, _INT]
    n, rp, ci, v = _csr(A)
    x = _c(x, np.float64)
    out = np.zeros(n) if y is None else np.array(y, dtype=np.float64, copy=True)
    _omp.orc_spmv_csr_omp(n, _p(rp), _p(ci), _p(v), _p(x), alpha, beta, _p(out), int(threads))
    return out


def spmm_csr(A, X, alpha=1.0, beta=0.0, Y=None):
    """Y = alpha A X + beta Y for row-major dense blocks X (n_cols x k)."""
    n, rp, ci, v = _csr(A)
    X = _c(X, np.float64)
    k = X.shape[1]
    Y = np.zeros((n, k)) if Y is None else np.array(Y, dtype=np.float64, copy=True, order="C")
    lib().orc_spmm_csr(n, _p(rp), _p(ci), _p(v), k, _p(X), k, alpha, beta, _p(Y), k)
    return Y


def spmv_dot2(A, x, alpha=1.0, beta=0.0, y=None):
    """Compensated (Dot2) reference of spmv_csr and the per-entry magnitude
    |alpha| |A| |x| + |beta| |y|.  Returns (y_ref, mag)."""
    n, rp, ci, v = _csr(A)
    x = _c(x, np.float64)
    yin = None if y is None else _c(y, np.float64)
    out, mag = np.zeros(n), np.zeros(n)
    lib().orc_spmv_csr_dot2(n, _p(rp), _p(ci), _p(v), _p(x), alpha, beta, _p(yin), _p(out),
                            _p(mag))
    return out, mag


def spmv_coo(n, coo, x, alpha=1.0, beta=0.0, y=None):
    x = _c(x, np.float64)
    out = np.zeros(n) if y is None else np.array(y, dtype=np.float64, copy=True)
    lib().orc_spmv_coo(n, len(coo["val"]), _p(coo["row"]), _p(coo["col"]), _p(coo["val"]),
                       _p(x), alpha, beta, _p(out))
    return out


def spmv_ell(n, ell, x, alpha=1.0, beta=0.0, y=None):
    x = _c(x, np.float64)
    out = np.zeros(n) if y is None else np.array(y, dtype=np.float64, copy=True)
    lib().orc_spmv_ell(n, ell["n_pad"], ell["K"], _p(ell["col"]), _p(ell["val"]), _p(x),
                       alpha, beta, _p(out))
    return out


def spmv_sellp(n, s, x, alpha=1.0, beta=0.0, y=None):
    x = _c(x, np.float64)
    out = np.zeros(n) if y is None else np.array(y, dtype=np.float64, copy=True)
    lib().orc_spmv_sellp(n, s["S"], _p(s["slice_len"]), _p(s["slice_set"]), _p(s["col"]),
                         _p(s["val"]), _p(x), alpha, beta, _p(out))
    return out


def spmv_hybrid(n, h, x, alpha=1.0, beta=0.0, y=None):
    x = _c(x, np.float64)
    out = np.zeros(n) if y is None else np.array(y, dtype=np.float64, copy=True)
    lib().orc_spmv_hybrid(n, h["n_pad"], h["K"], _p(h["ell_col"]), _p(h["ell_val"]),
                          len(h["coo_val"]), _p(h["coo_row"]), _p(h["coo_col"]),
                          _p(h["coo_val"]), _p(x), alpha, beta, _p(out))
    return out


# ----------------------------------------------------------- conversions

def to_coo(A):
    n, rp, ci, v = _csr(A)
    nnz = int(rp[n]) if n else 0
    row, col, val = np.empty(nnz, np.int32), np.empty(nnz, np.int32), np.empty(nnz)
    lib().orc_csr_to_coo(n, _p(rp), _p(ci), _p(v), _p(row), _p(col), _p(val))
    return dict(row=row, col=col, val=val)


def coo_to_csr(n, coo, n_cols):
    nnz = len(coo["val"])
    rp, ci, v = np.empty(n + 1, np.int32), np.empty(nnz, np.int32), np.empty(nnz)
    lib().orc_coo_to_csr(n, nnz, _p(_c(coo["row"], np.int32)), _p(_c(coo["col"], np.int32)),
                         _p(_c(coo["val"], np.float64)), _p(rp), _p(ci), _p(v))
    return dict(n_rows=n, n_cols=n_cols, row_ptr=rp, col_idx=ci, val=v)


def max_row_len(A):
    n, rp, _, _ = _csr(A)
    return int(lib().orc_max_row_len(n, _p(rp)))


def ell_n_pad(n):
    return int(lib().orc_ell_n_pad(n))


def to_ell(A, K=None):
    n, rp, ci, v = _csr(A)
    K = max_row_len(A) if K is None else K
    n_pad = ell_n_pad(n)
    col, val = np.empty(K * n_pad, np.int32), np.empty(K * n_pad)
    lib().orc_csr_to_ell(n, n_pad, K, _p(rp), _p(ci), _p(v), _p(col), _p(val))
    return dict(n_pad=n_pad, K=K, col=col, val=val)


def _nnz_of_padded(col):
    return int(np.count_nonzero(col >= 0))


def ell_to_csr(n, ell, n_cols):
    nnz = _nnz_of_padded(ell["col"])
    rp, ci, v = np.empty(n + 1, np.int32), np.empty(nnz, np.int32), np.empty(nnz)
    lib().orc_ell_to_csr(n, ell["n_pad"], ell["K"], _p(_c(ell["col"], np.int32)),
                         _p(_c(ell["val"], np.float64)), _p(rp), _p(ci), _p(v))
    return dict(n_rows=n, n_cols=n_cols, row_ptr=rp, col_idx=ci, val=v)


def to_sellp(A, S=64, f=1):
    n, rp, ci, v = _csr(A)
    ns = (n + S - 1) // S
    slen, sset = np.empty(ns, np.int32), np.empty(ns + 1, np.int32)
    total = int(lib().orc_sellp_sizes(n, _p(rp), S, f, _p(slen), _p(sset)))
    col, val = np.empty(total, np.int32), np.empty(total)
    lib().orc_csr_to_sellp(n, S, _p(rp), _p(ci), _p(v), _p(slen), _p(sset), _p(col), _p(val))
    return dict(S=S, f=f, slice_len=slen, slice_set=sset, col=col, val=val)


def sellp_to_csr(n, s, n_cols):
    nnz = _nnz_of_padded(s["col"])
    rp, ci, v = np.empty(n + 1, np.int32), np.empty(nnz, np.int32), np.empty(nnz)
    lib().orc_sellp_to_csr(n, s["S"], _p(s["slice_len"]), _p(s["slice_set"]),
                           _p(_c(s["col"], np.int32)), _p(_c(s["val"], np.float64)), _p(rp),
                           _p(ci), _p(v))
    return dict(n_rows=n, n_cols=n_cols, row_ptr=rp, col_idx=ci, val=v)


def hybrid_width(A, s_v=8):
    n, rp, _, _ = _csr(A)
    return int(lib().orc_hybrid_width(n, _p(rp), s_v))


def to_hybrid(A, K=None, s_v=8):
    n, rp, ci, v = _csr(A)
    K = hybrid_width(A, s_v) if K is None else K
    n_pad = ell_n_pad(n)
    over = int(lib().orc_hybrid_coo_nnz(n, _p(rp), K))
    ec, ev = np.empty(K * n_pad, np.int32), np.empty(K * n_pad)
    cr, cc, cv = np.empty(over, np.int32), np.empty(over, np.int32), np.empty(over)
    lib().orc_csr_to_hybrid(n, n_pad, K, _p(rp), _p(ci), _p(v), _p(ec), _p(ev), _p(cr), _p(cc),
                            _p(cv))
    return dict(n_pad=n_pad, K=K, ell_col=ec, ell_val=ev, coo_row=cr, coo_col=cc, coo_val=cv)


def hybrid_to_csr(n, h, n_cols):
    nnz = _nnz_of_padded(h["ell_col"]) + len(h["coo_val"])
    rp, ci, v = np.empty(n + 1, np.int32), np.empty(nnz, np.int32), np.empty(nnz)
    lib().orc_hybrid_to_csr(n, h["n_pad"], h["K"], _p(_c(h["ell_col"], np.int32)),
                            _p(_c(h["ell_val"], np.float64)), len(h["coo_val"]),
                            _p(_c(h["coo_row"], np.int32)), _p(_c(h["coo_col"], np.int32)),
                            _p(_c(h["coo_val"], np.float64)), _p(rp), _p(ci), _p(v))
    return dict(n_rows=n, n_cols=n_cols, row_ptr=rp, col_idx=ci, val=v)


# ---------------------------------------------------------------- BLAS-1

def dot(a, b):
    a, b = _c(a, np.float64), _c(b, np.float64)
    return float(lib().orc_dot(len(a), _p(a), _p(b)))


def dot2(a, b):
    a, b = _c(a, np.float64), _c(b, np.float64)
    return float(lib().orc_dot2(len(a), _p(a), _p(b)))


def true_rel_residual(A, b, x):
    n, rp, ci, v = _csr(A)
    b, x = _c(b, np.float64), _c(x, np.float64)
    return float(lib().orc_true_rel_residual(n, _p(rp), _p(ci), _p(v), _p(b), _p(x)))


# ------------------------------------------------------------------- CG

def cg(A, b, x0=None, tol=1e-10, maxit=10000):
    """Hestenes-Stiefel CG.  Returns (x, status, iterations, true rel. residual)."""
    n, rp, ci, v = _csr(A)
    b = _c(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it, res = C.c_int(0), C.c_double(0.0)
    st = lib().orc_cg(n, _p(rp), _p(ci), _p(v), _p(b), _p(x), tol, maxit, C.byref(it),
                      C.byref(res))
    return x, int(st), it.value, res.value


def cg_single_reduction(A, b, x0=None, tol=1e-10, maxit=10000):
    """Chronopoulos-Gear single-reduction CG.  Returns (x, status, iterations,
    true rel. residual)."""
    n, rp, ci, v = _csr(A)
    b = _c(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it, res = C.c_int(0), C.c_double(0.0)
    st = lib().orc_cg_single_reduction(n, _p(rp), _p(ci), _p(v), _p(b), _p(x), tol, maxit, C.byref(it),
                                       C.byref(res))
    return x, int(st), it.value, res.value


def pcg_jacobi(A, b, x0=None, tol=1e-10, maxit=10000):
    """CG preconditioned by diag(A).  Returns (x, status, iterations, true
    rel. residual)."""
    n, rp, ci, v = _csr(A)
    b = _c(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it, res = C.c_int(0), C.c_double(0.0)
    st = lib().orc_pcg_jacobi(n, _p(rp), _p(ci), _p(v), _p(b), _p(x), tol, maxit, C.byref(it), C.byref(res))
    return x, int(st), it.value, res.value


def bj_blocks(A, max_bs):
    """Block boundaries of the block-Jacobi preconditioner (supervariables
    of identical column lists, cut at max_bs rows, merged greedily up to
    max_bs rows): int32 array of n_blocks + 1 row offsets."""
    n, rp, ci, _ = _csr(A)
    bp = np.zeros(n + 1, dtype=np.int32)
    nb = C.c_int64(0)
    st = lib().orc_bj_blocks(n, _p(rp), _p(ci), int(max_bs), _p(bp), C.byref(nb))
    if st != OK:
        raise ValueError("max_bs must be in 1..32")
    return bp[:nb.value + 1].copy()


def bj_invert(A, block_ptr, max_bs):
    """Inverses of the diagonal blocks, n * max_bs doubles: entry (i, j) of
    the block starting at row o with s rows at o * max_bs + j * s + i.
    Returns (status, inv); status BREAKDOWN for a singular block."""
    n, rp, ci, v = _csr(A)
    bp = _c(block_ptr, np.int32)
    inv = np.zeros(max(n, 1) * max_bs)
    st = lib().orc_bj_invert(n, _p(rp), _p(ci), _p(v), int(max_bs), _p(bp), len(bp) - 1, _p(inv))
    return int(st), inv[:n * max_bs]


def bj_apply(block_ptr, max_bs, inv, r):
    """z = M^-1 r with the inverses of bj_invert."""
    bp = _c(block_ptr, np.int32)
    r = _c(r, np.float64)
    z = np.zeros(len(r))
    inv = _c(inv, np.float64)
    lib().orc_bj_apply(int(max_bs), _p(bp), len(bp) - 1, _p(inv), _p(r), _p(z))
    return z


def pcg_block_jacobi(A, b, max_bs, x0=None, tol=1e-10, maxit=10000):
    """CG preconditioned by block-Jacobi with blocks of at most max_bs rows.
    Returns (x, status, iterations, true rel. residual)."""
    n, rp, ci, v = _csr(A)
    b = _c(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it, res = C.c_int(0), C.c_double(0.0)
    st = lib().orc_pcg_block_jacobi(n, _p(rp), _p(ci), _p(v), int(max_bs), _p(b), _p(x), tol, maxit,
                                    C.byref(it), C.byref(res))
    return x, int(st), it.value, res.value


def bicgstab(A, b, x0=None, tol=1e-10, maxit=10000):
    """BiCGSTAB (van der Vorst).  Returns (x, status, steps, true rel. residual)."""
    n, rp, ci, v = _csr(A)
    b = _c(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it, res = C.c_int(0), C.c_double(0.0)
    st = lib().orc_bicgstab(n, _p(rp), _p(ci), _p(v), _p(b), _p(x), tol, maxit, C.byref(it), C.byref(res))
    return x, int(st), it.value, res.value


def gmres(A, b, x0=None, tol=1e-10, restart=30, maxit=10000):
    """Restarted GMRES(restart).  Returns (x, status, Arnoldi steps, true
    rel. residual)."""
    n, rp, ci, v = _csr(A)
    b = _c(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it, res = C.c_int(0), C.c_double(0.0)
    st = lib().orc_gmres(n, _p(rp), _p(ci), _p(v), _p(b), _p(x), tol, restart, maxit, C.byref(it), C.byref(res))
    return x, int(st), it.value, res.value


def cg_batched(B, b, tol=1e-10, maxit=10000):
    """CG on every system of a ``synthetic.batched_spd`` batch.
    Returns (x, status[count], iterations[count], rel_res[count])."""
    count = len(B["sizes"])
    rp, ci, v = _c(B["row_ptr"], np.int32), _c(B["col_idx"], np.int32), _c(B["val"], np.float64)
    ro = _c(B["row_off"], np.int64)
    b = _c(b, np.float64)
    x = np.zeros(len(b))
    it, res, st = np.zeros(count, np.int32), np.zeros(count), np.zeros(count, np.int32)
    lib().orc_cg_batched(count, _p(ro), _p(rp), _p(ci), _p(v), _p(b), _p(x), tol, maxit, _p(it),
                         _p(res), _p(st))
    return x, st, it, res


def round_bf16(v, up=False):
    return float(lib().orc_round_bf16(float(v), int(up)))


def round_fp32(v, up=False):
    return float(lib().orc_round_fp32(float(v), int(up)))


def round_matrix(A, prec):
    """Values of the low-precision copy (prec 'fp32' or 'bf16') as float64."""
    n, rp, ci, v = _csr(A)
    out = np.empty_like(v)
    lib().orc_round_matrix(n, _p(rp), _p(ci), _p(v), 2 if prec == "bf16" else 1, _p(out))
    return out


def cg_mixed(A, b, prec="fp32", x0=None, tol=1e-10, maxit_outer=100, inner_tol=1e-4,
             inner_maxit=100000, precond="none"):
    """Mixed-precision CG with FP64 refinement (precond "jacobi": the inner
    CG preconditioned by the diagonal of the rounded matrix).
    Returns (x, status, outer corrections, inner iterations, true rel. residual)."""
    n, rp, ci, v = _csr(A)
    vlo = round_matrix(A, prec)
    b = _c(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    o, i, res = C.c_int(0), C.c_int(0), C.c_double(0.0)
    if precond == "jacobi":
        st = lib().orc_cg_mixed_precond(n, _p(rp), _p(ci), _p(v), _p(vlo), _p(b), _p(x), tol, maxit_outer,
                                        inner_tol, inner_maxit, 1, C.byref(o), C.byref(i), C.byref(res))
    else:
        st = lib().orc_cg_mixed(n, _p(rp), _p(ci), _p(v), _p(vlo), _p(b), _p(x), tol, maxit_outer,
                                inner_tol, inner_maxit, C.byref(o), C.byref(i), C.byref(res))
    return x, int(st), o.value, i.value, res.value


def cholesky_solve(Ad, b):
    Ad = _c(Ad, np.float64)
    b = _c(b, np.float64)
    n = len(b)
    x = np.zeros(n)
    st = lib().orc_cholesky_solve(n, _p(Ad), _p(b), _p(x))
    return x, int(st)


def features(A):
    """The 12 selector statistics (see oracle.c, orc_features)."""
    n, rp, ci, _ = _csr(A)
    f = np.zeros(12)
    lib().orc_features(n, _p(rp), _p(ci), _p(f))
    return f


def to_dense(A):
    """Dense copy of a small CSR matrix (test helper; no arithmetic)."""
    n, m = int(A["n_rows"]), int(A["n_cols"])
    D = np.zeros((n, m))
    rp = A["row_ptr"]
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            D[i, A["col_idx"][k]] = A["val"][k]
    return D
