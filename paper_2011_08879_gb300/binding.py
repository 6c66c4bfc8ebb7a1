"""ctypes binding of libgkogb.so (include/gko_gb300.h), argument marshalling only.

Every ``gko_*`` function here has the name, argument order and meaning of
the C entry point it wraps.  Pointers are passed as Python ints (e.g. a
torch tensor's ``data_ptr()``), streams as ``torch.cuda.Stream.cuda_stream``
ints (0 = legacy default stream).  A non-zero status raises GkoError with
the library's message, except where noted.  There is no fallback: if the
library is missing or cannot be loaded, importing raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgkogb.so")
LIB_CHECKED_PATH = os.path.join(HERE, "libgkogb_checked.so")

# formats
FMT_CSR, FMT_COO, FMT_ELL, FMT_SELLP, FMT_HYBRID, FMT_AUTO = range(6)
FORMATS = {"csr": FMT_CSR, "coo": FMT_COO, "ell": FMT_ELL, "sellp": FMT_SELLP, "hybrid": FMT_HYBRID,
           "auto": FMT_AUTO}
# status codes
(OK, ERR_INVALID_ARG, ERR_DIM_MISMATCH, ERR_FORMAT_UNAVAILABLE, ERR_FORMAT_TOO_LARGE, ERR_OUT_OF_MEMORY,
 ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_INVALID_MATRIX, ERR_TIMEOUT, ERR_CUDA) = range(11)
# value types
F64, F32, BF16 = 0, 1, 2
# batched-CG layout flags (OR'ed with the block size)
BATCH_SHARED_P, BATCH_SHARED_PQ = 0x10000, 0x20000


def batch_layout(code: int) -> str:
    """Readable name of a gko_cg_batched block_size code."""
    if code == 0:
        return "autotuned"
    if code < 0:
        return "registers/%d" % -code
    if code & BATCH_SHARED_P:
        return "shared_p/%d" % (code & 0xFFFF)
    if code & BATCH_SHARED_PQ:
        return "shared_pq/%d" % (code & 0xFFFF)
    return "shared_xrpq/%d" % code


def batch_layout_code(name: str) -> int:
    """Inverse of batch_layout: "shared_p/128" -> BATCH_SHARED_P | 128."""
    kind, _, bs = name.partition("/")
    flags = {"shared_p": BATCH_SHARED_P, "shared_pq": BATCH_SHARED_PQ, "shared_xrpq": 0, "registers": -1}
    if kind == "autotuned" and not bs:
        return 0
    if kind not in flags or not bs.isdigit():
        raise ValueError("unknown batched layout %r" % name)
    return -int(bs) if flags[kind] == -1 else flags[kind] | int(bs)


# kernel configurations
(CFG_DEFAULT, CFG_CSR_SUBWARP_1, CFG_CSR_SUBWARP_2, CFG_CSR_SUBWARP_4, CFG_CSR_SUBWARP_8, CFG_CSR_SUBWARP_16,
 CFG_CSR_SUBWARP_32, CFG_CSR_NNZSPLIT, CFG_CSR_BANDED, CFG_CSR_ROWBLOCK, CFG_CSR_BINNED) = range(11)


class GkoError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__("%s: %s (%s)" % (where, msg, status_name(status)))
        self.status = status


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("outer_iterations", C.c_int32), ("rel_residual", C.c_double),
                ("status", C.c_int32), ("aux", C.c_int32)]


_P, _I64, _I32, _D, _F, _INT, _U32P = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_float, C.c_int, C.c_void_p

_SIGS = {
    "gko_last_error": (C.c_char_p, []),
    "gko_status_string": (C.c_char_p, [_INT]),
    "gko_version": (C.c_char_p, []),
    "gko_set_wait_limit": (_INT, [C.c_uint32]),
    "gko_measure_ceilings": (_INT, [_P, _P, _P, _I64, _P]),
    "gko_matrix_create_csr": (_INT, [_I64, _I64, _I64, _P, _P, _P, _INT, _P, C.POINTER(_P)]),
    "gko_matrix_destroy": (_INT, [_P]),
    "gko_matrix_set_params": (_INT, [_P, _INT, _INT, _D]),
    "gko_convert": (_INT, [_P, _INT, _INT, _P]),
    "gko_matrix_release": (_INT, [_P, _INT]),
    "gko_matrix_info": (_INT, [_P, _INT, _P]),
    "gko_matrix_export": (_INT, [_P, _INT, _INT, _P, _I64, _INT, _P]),
    "gko_matrix_errors": (_INT, [_P, _P, _INT, _P]),
    "gko_spmv": (_INT, [_INT, _P, _P, _P, _D, _D, _P]),
    "gko_spmv_config": (_INT, [_INT, _INT, _P, _P, _P, _D, _D, _P]),
    "gko_spmv_host": (_INT, [_INT, _P, _P, _P, _D, _D, _P]),
    "gko_spmv_coo_noalloc": (_INT, [_I64, _I64, _I64, _P, _P, _P, _P, _P, _D, _D, _P, _P]),
    "gko_cg": (_INT, [_P, _INT, _P, _P, _D, _INT, _P, C.POINTER(SolveInfo)]),
    "gko_cg_single_reduction": (_INT, [_P, _INT, _P, _P, _D, _INT, _P, C.POINTER(SolveInfo)]),
    "gko_pcg_jacobi": (_INT, [_P, _INT, _P, _P, _D, _INT, _P, C.POINTER(SolveInfo)]),
    "gko_bicgstab": (_INT, [_P, _INT, _P, _P, _D, _INT, _P, C.POINTER(SolveInfo)]),
    "gko_cg_multi": (_INT, [_P, _I64, _P, _I64, _P, _I64, _D, _INT, _P, _P]),
    "gko_block_jacobi_create": (_INT, [_P, _INT, _P, C.POINTER(_P)]),
    "gko_block_jacobi_destroy": (_INT, [_P]),
    "gko_block_jacobi_export": (_INT, [_P, C.POINTER(_I64), _P, _P, _P]),
    "gko_block_jacobi_apply": (_INT, [_P, _P, _P, _P]),
    "gko_pcg_block_jacobi": (_INT, [_P, _INT, _P, _P, _P, _D, _INT, _P, C.POINTER(SolveInfo)]),
    "gko_spmm": (_INT, [_P, _I64, _P, _I64, _P, _I64, _D, _D, _P]),
    "gko_gmres": (_INT, [_P, _INT, _P, _P, _D, _INT, _INT, _P, C.POINTER(SolveInfo)]),
    "gko_cg_mixed_precond": (_INT, [_P, _INT, _INT, _P, _P, _D, _INT, _D, _INT, _P, C.POINTER(SolveInfo)]),
    "gko_cg_mixed": (_INT, [_P, _INT, _P, _P, _D, _INT, _D, _INT, _P, C.POINTER(SolveInfo)]),
    "gko_batch_create": (_INT, [_I64, _P, _P, _P, _P, _INT, _P, C.POINTER(_P)]),
    "gko_batch_destroy": (_INT, [_P]),
    "gko_cg_batched": (_INT, [_P, _P, _P, _D, _INT, _INT, _P, _P]),
    "gko_batch_autotune": (_INT, [_P, _P, _P, _D, _INT, _P, C.POINTER(_INT)]),
    "gko_features": (_INT, [_P, _P, _P]),
    "gko_mlp_param_count": (_I64, [_INT]),
    "gko_mlp_forward": (_INT, [_P, _INT, _P, _INT, _P, _P]),
    "gko_mlp_grad": (_INT, [_P, _INT, _P, _P, _P, _INT, _P, _P, _P]),
    "gko_mlp_adam": (_INT, [_P, _P, _P, _P, _I64, _INT, _F, _F, _F, _F, _P]),
    "gko_selector_load": (_INT, [_P, _INT, _P, _P, _P, _P]),
    "gko_select_format": (_INT, [_P, C.POINTER(_INT), C.POINTER(_INT), _P]),
    "gko_selector_clear": (_INT, []),
    "gko_autotune_format": (_INT, [_P, C.POINTER(_INT), C.POINTER(_INT), _P, _P]),
}


def _load(path=LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError("%s is not built; run paper_2011_08879_gb300.build.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()
_checked = None


def checked_lib() -> C.CDLL:
    """The bounds-checked copy of the library (built with GKO_CHECK_BOUNDS:
    unvalidated indices are clamped and reported as error bit 1), loaded on
    first use; same entry points and signatures as ``lib``."""
    global _checked
    if _checked is None:
        _checked = _load(LIB_CHECKED_PATH)
    return _checked


def status_name(s: int) -> str:
    return lib.gko_status_string(int(s)).decode()


def last_error() -> str:
    return lib.gko_last_error().decode()


def _check(status: int, where: str, allow=()) -> int:
    if status != OK and status not in allow:
        raise GkoError(status, where, last_error())
    return status


def gko_version() -> str:
    return lib.gko_version().decode()


def gko_set_wait_limit(polls) -> None:
    """Poll limit of the staged kernels' first bounded wait (tests of the
    timeout path); 0xFFFFFFFF restores the default."""
    _check(lib.gko_set_wait_limit(polls), "gko_set_wait_limit")


def gko_matrix_create_csr(n_rows, n_cols, nnz, row_ptr, col, val, on_device, stream=0) -> int:
    out = _P()
    _check(lib.gko_matrix_create_csr(n_rows, n_cols, nnz, row_ptr, col, val, int(on_device), stream, C.byref(out)),
           "gko_matrix_create_csr")
    return out.value


def gko_matrix_destroy(A) -> None:
    _check(lib.gko_matrix_destroy(A), "gko_matrix_destroy")


def gko_matrix_set_params(A, sellp_slice=0, sellp_stride=0, ell_factor=0.0) -> None:
    _check(lib.gko_matrix_set_params(A, sellp_slice, sellp_stride, ell_factor), "gko_matrix_set_params")


def gko_convert(A, src, dst, stream=0) -> None:
    _check(lib.gko_convert(A, src, dst, stream), "gko_convert")


def gko_matrix_release(A, fmt) -> None:
    _check(lib.gko_matrix_release(A, fmt), "gko_matrix_release")


def gko_matrix_info(A, fmt) -> list:
    info = (C.c_int64 * 8)()
    _check(lib.gko_matrix_info(A, fmt, info), "gko_matrix_info")
    return list(info)


def gko_matrix_export(A, fmt, array, dst, nbytes, to_host, stream=0) -> None:
    _check(lib.gko_matrix_export(A, fmt, array, dst, nbytes, int(to_host), stream), "gko_matrix_export")


def gko_matrix_errors(A, clear=False, stream=0) -> int:
    bits = C.c_uint32(0)
    _check(lib.gko_matrix_errors(A, C.byref(bits), int(clear), stream), "gko_matrix_errors")
    return bits.value


def gko_spmv(fmt, A, x, y, alpha=1.0, beta=0.0, stream=0) -> None:
    _check(lib.gko_spmv(fmt, A, x, y, alpha, beta, stream), "gko_spmv")


def gko_spmv_config(fmt, config, A, x, y, alpha=1.0, beta=0.0, stream=0) -> None:
    _check(lib.gko_spmv_config(fmt, config, A, x, y, alpha, beta, stream), "gko_spmv_config")


def gko_spmv_host(fmt, A, x_host, y_host, alpha=1.0, beta=0.0, stream=0) -> None:
    _check(lib.gko_spmv_host(fmt, A, x_host, y_host, alpha, beta, stream), "gko_spmv_host")


def gko_spmv_coo_noalloc(n_rows, n_cols, nnz, row, col, val, x, y, alpha=1.0, beta=0.0, err_flags=None,
                         stream=0) -> None:
    """COO SpMV without any allocation (see the header); device pointers."""
    _check(lib.gko_spmv_coo_noalloc(n_rows, n_cols, nnz, row, col, val, x, y, alpha, beta, err_flags, stream),
           "gko_spmv_coo_noalloc")


def gko_cg(A, fmt, b, x, tol, maxit, stream=0, raise_on=()) -> SolveInfo:
    """Returns the SolveInfo; NOT_CONVERGED and BREAKDOWN are reported in
    info.status (not raised) unless listed in raise_on."""
    info = SolveInfo()
    s = lib.gko_cg(A, fmt, b, x, tol, maxit, stream, C.byref(info))
    allow = tuple(c for c in (ERR_NOT_CONVERGED, ERR_BREAKDOWN) if c not in raise_on)
    _check(s, "gko_cg", allow)
    info.status = s
    return info


def gko_cg_single_reduction(A, fmt, b, x, tol, maxit, stream=0, raise_on=()) -> SolveInfo:
    """As gko_cg, for the single-reduction (Chronopoulos-Gear) CG."""
    info = SolveInfo()
    s = lib.gko_cg_single_reduction(A, fmt, b, x, tol, maxit, stream, C.byref(info))
    allow = tuple(c for c in (ERR_NOT_CONVERGED, ERR_BREAKDOWN) if c not in raise_on)
    _check(s, "gko_cg_single_reduction", allow)
    info.status = s
    return info


def gko_pcg_jacobi(A, fmt, b, x, tol, maxit, stream=0, raise_on=()) -> SolveInfo:
    """As gko_cg, preconditioned by the diagonal of A."""
    info = SolveInfo()
    s = lib.gko_pcg_jacobi(A, fmt, b, x, tol, maxit, stream, C.byref(info))
    allow = tuple(c for c in (ERR_NOT_CONVERGED, ERR_BREAKDOWN) if c not in raise_on)
    _check(s, "gko_pcg_jacobi", allow)
    info.status = s
    return info


def gko_cg_multi(A, k, B, ldb, X, ldx, tol, maxit, stream=0, infos=None) -> int:
    """infos: optional ctypes array of k SolveInfo.  Returns the status
    (NOT_CONVERGED / BREAKDOWN of a column are not raised)."""
    s = lib.gko_cg_multi(A, k, B, ldb, X, ldx, tol, maxit, stream, infos)
    _check(s, "gko_cg_multi", (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
    return s


def gko_block_jacobi_create(A, max_block_size, stream=0) -> int:
    out = _P()
    _check(lib.gko_block_jacobi_create(A, max_block_size, stream, C.byref(out)), "gko_block_jacobi_create")
    return out.value


def gko_block_jacobi_destroy(M) -> None:
    _check(lib.gko_block_jacobi_destroy(M), "gko_block_jacobi_destroy")


def gko_block_jacobi_export(M, block_ptr=None, inv=None, stream=0) -> int:
    """Returns n_blocks; fills the host buffers block_ptr / inv when given."""
    nb = _I64(0)
    _check(lib.gko_block_jacobi_export(M, C.byref(nb), block_ptr, inv, stream), "gko_block_jacobi_export")
    return nb.value


def gko_block_jacobi_apply(M, r, z, stream=0) -> None:
    _check(lib.gko_block_jacobi_apply(M, r, z, stream), "gko_block_jacobi_apply")


def gko_pcg_block_jacobi(A, fmt, M, b, x, tol, maxit, stream=0, raise_on=()) -> SolveInfo:
    """As gko_pcg_jacobi, preconditioned by the block-Jacobi object M."""
    info = SolveInfo()
    s = lib.gko_pcg_block_jacobi(A, fmt, M, b, x, tol, maxit, stream, C.byref(info))
    allow = tuple(c for c in (ERR_NOT_CONVERGED, ERR_BREAKDOWN) if c not in raise_on)
    _check(s, "gko_pcg_block_jacobi", allow)
    info.status = s
    return info


def gko_bicgstab(A, fmt, b, x, tol, maxit, stream=0, raise_on=()) -> SolveInfo:
    """BiCGSTAB; NOT_CONVERGED and BREAKDOWN are reported in info.status."""
    info = SolveInfo()
    s = lib.gko_bicgstab(A, fmt, b, x, tol, maxit, stream, C.byref(info))
    allow = tuple(c for c in (ERR_NOT_CONVERGED, ERR_BREAKDOWN) if c not in raise_on)
    _check(s, "gko_bicgstab", allow)
    info.status = s
    return info


def gko_spmm(A, k, x, ldx, y, ldy, alpha=1.0, beta=0.0, stream=0) -> None:
    """Y = alpha A X + beta Y (row-major blocks; device pointers)."""
    _check(lib.gko_spmm(A, k, x, ldx, y, ldy, alpha, beta, stream), "gko_spmm")


def gko_gmres(A, fmt, b, x, tol, restart, maxit, stream=0, raise_on=()) -> SolveInfo:
    """Restarted GMRES; NOT_CONVERGED and BREAKDOWN are reported in info.status."""
    info = SolveInfo()
    s = lib.gko_gmres(A, fmt, b, x, tol, restart, maxit, stream, C.byref(info))
    allow = tuple(c for c in (ERR_NOT_CONVERGED, ERR_BREAKDOWN) if c not in raise_on)
    _check(s, "gko_gmres", allow)
    info.status = s
    return info


def gko_cg_mixed(A, inner_dtype, b, x, tol, maxit_outer, inner_tol, inner_maxit, stream=0) -> SolveInfo:
    info = SolveInfo()
    s = lib.gko_cg_mixed(A, inner_dtype, b, x, tol, maxit_outer, inner_tol, inner_maxit, stream, C.byref(info))
    _check(s, "gko_cg_mixed", (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
    info.status = s
    return info


PRECOND_NONE, PRECOND_JACOBI = 0, 1


def gko_cg_mixed_precond(A, inner_dtype, precond, b, x, tol, maxit_outer, inner_tol, inner_maxit,
                         stream=0) -> SolveInfo:
    info = SolveInfo()
    s = lib.gko_cg_mixed_precond(A, inner_dtype, precond, b, x, tol, maxit_outer, inner_tol, inner_maxit, stream,
                                 C.byref(info))
    _check(s, "gko_cg_mixed_precond", (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
    info.status = s
    return info


def gko_batch_create(count, row_off, row_ptr, col, val, on_device, stream=0) -> int:
    out = _P()
    _check(lib.gko_batch_create(count, row_off, row_ptr, col, val, int(on_device), stream, C.byref(out)),
           "gko_batch_create")
    return out.value


def gko_batch_destroy(B) -> None:
    _check(lib.gko_batch_destroy(B), "gko_batch_destroy")


def gko_cg_batched(B, b, x, tol, maxit, block_size=0, stream=0, infos=None) -> int:
    """infos: optional ctypes array of SolveInfo (count entries).  Returns the
    worst status (NOT_CONVERGED / BREAKDOWN are not raised)."""
    s = lib.gko_cg_batched(B, b, x, tol, maxit, block_size, stream, infos)
    _check(s, "gko_cg_batched", (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
    return s


def gko_batch_autotune(B, b, x, tol, maxit, stream=0) -> int:
    best = C.c_int(0)
    _check(lib.gko_batch_autotune(B, b, x, tol, maxit, stream, C.byref(best)), "gko_batch_autotune")
    return best.value


def gko_features(A, out_host, stream=0) -> None:
    _check(lib.gko_features(A, out_host, stream), "gko_features")


def gko_mlp_param_count(n_out) -> int:
    return int(lib.gko_mlp_param_count(n_out))


def gko_mlp_forward(params, n_out, X, batch, out, stream=0) -> None:
    _check(lib.gko_mlp_forward(params, n_out, X, batch, out, stream), "gko_mlp_forward")


def gko_mlp_grad(params, n_out, X, Y, M, batch, grad, loss, stream=0) -> None:
    _check(lib.gko_mlp_grad(params, n_out, X, Y, M, batch, grad, loss, stream), "gko_mlp_grad")


def gko_mlp_adam(params, grad, m, v, count, t, lr, beta1, beta2, eps, stream=0) -> None:
    _check(lib.gko_mlp_adam(params, grad, m, v, count, t, lr, beta1, beta2, eps, stream), "gko_mlp_adam")


def gko_selector_load(params_host, n_out, feat_mean, feat_scale, fmts, cfgs) -> None:
    _check(lib.gko_selector_load(params_host, n_out, feat_mean, feat_scale, fmts, cfgs), "gko_selector_load")


def gko_select_format(A, stream=0):
    f, c = C.c_int(0), C.c_int(0)
    _check(lib.gko_select_format(A, C.byref(f), C.byref(c), stream), "gko_select_format")
    return f.value, c.value


def gko_selector_clear() -> None:
    """Uninstall the selector (GKO_FMT_AUTO then autotunes exhaustively)."""
    _check(lib.gko_selector_clear(), "gko_selector_clear")


N_CANDIDATES = 10


def gko_autotune_format(A, stream=0):
    """(fmt, config, times_us) of the exhaustive autotuner (see the header)."""
    f, c = _INT(), _INT()
    times = (C.c_double * N_CANDIDATES)()
    _check(lib.gko_autotune_format(A, C.byref(f), C.byref(c), times, stream), "gko_autotune_format")
    return f.value, c.value, list(times)


def gko_measure_ceilings(gather_span=1 << 21, stream=0):
    """(FP64 TFMA/s, FP32 TFMA/s, random gathers G/s) of the running GPU."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(lib.gko_measure_ceilings(C.byref(a), C.byref(b), C.byref(c), int(gather_span), stream),
           "gko_measure_ceilings")
    return a.value, b.value, c.value
