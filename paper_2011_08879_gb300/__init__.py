"""GB300-native sparse hot path: SpMV (CSR, COO, ELL, SELL-P, hybrid), format
conversions, CG (FP64, mixed FP32/BF16 + FP64 refinement, batched) and a
learned format selector, all in hand-written sm_103a kernels behind the C ABI
of include/gko_gb300.h.

``binding`` holds the ctypes functions with the C names; ``Matrix`` and
``Batch`` below only marshal torch tensors / numpy arrays into those calls.
Importing fails loudly when the CUDA library has not been built.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding
from .binding import *  # noqa: F401,F403  (gko_* entry points and constants)
from .binding import FORMATS, GkoError, SolveInfo


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _dev_f64(t, n, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    if t.numel() != n:
        raise ValueError("%s has %d entries, expected %d" % (name, t.numel(), n))
    return t.data_ptr()


def _fmt(f):
    return FORMATS[f] if isinstance(f, str) else int(f)


class Matrix:
    """Owning wrapper of a gko_matrix handle built from a CSR matrix.

    ``csr`` is a dict with n_rows, n_cols, row_ptr, col_idx, val (numpy
    arrays on the host, or CUDA tensors with on_device=True)."""

    def __init__(self, csr, stream=None, on_device=False):
        self.n_rows, self.n_cols = int(csr["n_rows"]), int(csr["n_cols"])
        st = _stream(stream)
        if on_device:
            rp, ci, v = csr["row_ptr"], csr["col_idx"], csr["val"]
            self.nnz = int(ci.numel())
            ptrs = (rp.data_ptr(), ci.data_ptr() if self.nnz else None, v.data_ptr() if self.nnz else None)
        else:
            rp = np.ascontiguousarray(csr["row_ptr"], dtype=np.int32)
            ci = np.ascontiguousarray(csr["col_idx"], dtype=np.int32)
            v = np.ascontiguousarray(csr["val"], dtype=np.float64)
            self.nnz = int(len(ci))
            ptrs = (rp.ctypes.data, ci.ctypes.data if self.nnz else None, v.ctypes.data if self.nnz else None)
        self.handle = None
        self.handle = binding.gko_matrix_create_csr(self.n_rows, self.n_cols, self.nnz, *ptrs, on_device, st)

    def close(self):
        if self.handle:
            binding.gko_matrix_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, sellp_slice=0, sellp_stride=0, ell_factor=0.0):
        binding.gko_matrix_set_params(self.handle, sellp_slice, sellp_stride, ell_factor)

    def convert(self, dst, src="csr", stream=None):
        binding.gko_convert(self.handle, _fmt(src), _fmt(dst), _stream(stream))

    def release(self, fmt):
        binding.gko_matrix_release(self.handle, _fmt(fmt))

    def info(self, fmt):
        return binding.gko_matrix_info(self.handle, _fmt(fmt))

    def has(self, fmt):
        return bool(self.info(fmt)[0])

    _ARRAYS = {
        FORMATS["csr"]: (("row_ptr", np.int32), ("col", np.int32), ("val", np.float64)),
        FORMATS["coo"]: (("row", np.int32), ("col", np.int32), ("val", np.float64)),
        FORMATS["ell"]: (("col", np.int32), ("val", np.float64)),
        FORMATS["sellp"]: (("slice_len", np.int32), ("slice_set", np.int32), ("col", np.int32),
                           ("val", np.float64)),
        FORMATS["hybrid"]: (("ell_col", np.int32), ("ell_val", np.float64), ("coo_row", np.int32),
                            ("coo_col", np.int32), ("coo_val", np.float64)),
    }

    def _sizes(self, f):
        info = self.info(f)
        n, nnz = self.n_rows, self.nnz
        if f == FORMATS["csr"]:
            return [n + 1, nnz, nnz]
        if f == FORMATS["coo"]:
            return [nnz, nnz, nnz]
        if f == FORMATS["ell"]:
            return [info[6], info[6]]
        if f == FORMATS["sellp"]:
            return [info[5], info[5] + 1, info[6], info[6]]
        slots = info[4] * info[5]
        return [slots, slots, info[6], info[6], info[6]]

    def export(self, fmt, stream=None):
        """All arrays of a materialised format as host numpy arrays (dict)."""
        f = _fmt(fmt)
        out = {}
        for i, ((name, dt), cnt) in enumerate(zip(self._ARRAYS[f], self._sizes(f))):
            a = np.empty(int(cnt), dtype=dt)
            binding.gko_matrix_export(self.handle, f, i, a.ctypes.data if a.size else None, a.nbytes, True,
                                      _stream(stream))
            out[name] = a
        info = self.info(f)
        out["info"] = info
        return out

    def errors(self, clear=False, stream=None):
        return binding.gko_matrix_errors(self.handle, clear, _stream(stream))

    def spmv(self, x, y, alpha=1.0, beta=0.0, fmt="csr", config=0, stream=None):
        xp = _dev_f64(x, self.n_cols, "x")
        yp = _dev_f64(y, self.n_rows, "y")
        if config:
            binding.gko_spmv_config(_fmt(fmt), config, self.handle, xp, yp, alpha, beta, _stream(stream))
        else:
            binding.gko_spmv(_fmt(fmt), self.handle, xp, yp, alpha, beta, _stream(stream))
        return y

    def spmm(self, X, Y, alpha=1.0, beta=0.0, stream=None):
        """Y = alpha A X + beta Y; X (n_cols x k), Y (n_rows x k): row-major
        (C-contiguous) float64 CUDA tensors."""
        import torch
        for t, rows, name in ((X, self.n_cols, "X"), (Y, self.n_rows, "Y")):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2
                    and t.is_contiguous() and t.shape[0] == rows):
                raise TypeError("%s must be a contiguous float64 CUDA tensor with %d rows" % (name, rows))
        if X.shape[1] != Y.shape[1]:
            raise ValueError("X and Y need the same number of columns")
        k = X.shape[1]
        binding.gko_spmm(self.handle, k, X.data_ptr(), max(k, 1), Y.data_ptr(), max(k, 1), alpha, beta,
                         _stream(stream))
        return Y

    def spmv_host(self, x, y, alpha=1.0, beta=0.0, fmt="csr", stream=None):
        """x, y: host float64 arrays (numpy or pinned CPU tensors)."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        binding.gko_spmv_host(_fmt(fmt), self.handle, ptr(x), ptr(y), alpha, beta, _stream(stream))
        return y

    def cg(self, b, x, tol=1e-10, maxit=10000, fmt="csr", stream=None):
        return binding.gko_cg(self.handle, _fmt(fmt), _dev_f64(b, self.n_rows, "b"),
                              _dev_f64(x, self.n_rows, "x"), tol, maxit, _stream(stream))

    def cg_single_reduction(self, b, x, tol=1e-10, maxit=10000, fmt="csr", stream=None):
        return binding.gko_cg_single_reduction(self.handle, _fmt(fmt), _dev_f64(b, self.n_rows, "b"),
                                               _dev_f64(x, self.n_rows, "x"), tol, maxit, _stream(stream))

    def pcg_jacobi(self, b, x, tol=1e-10, maxit=10000, fmt="csr", stream=None):
        return binding.gko_pcg_jacobi(self.handle, _fmt(fmt), _dev_f64(b, self.n_rows, "b"),
                                      _dev_f64(x, self.n_rows, "x"), tol, maxit, _stream(stream))

    def cg_multi(self, B, X, tol=1e-10, maxit=10000, stream=None):
        """CG on A X = B for the k <= 32 columns of the row-major device
        blocks B, X (torch tensors of shape (n, k), last dimension
        contiguous; X holds the initial guess).  Returns (status, infos)."""
        import torch
        for t, name in ((B, "B"), (X, "X")):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2):
                raise TypeError("%s must be a 2-D float64 CUDA tensor" % name)
        k = int(B.shape[1])
        if tuple(B.shape) != (self.n_rows, k) or tuple(X.shape) != (self.n_rows, k):
            raise ValueError("B and X must be (n_rows, k)")
        if B.stride(1) != 1 or X.stride(1) != 1:
            raise ValueError("B and X need a contiguous last dimension")
        infos = (SolveInfo * k)()
        s = binding.gko_cg_multi(self.handle, k, B.data_ptr(), B.stride(0), X.data_ptr(), X.stride(0), tol, maxit,
                                 _stream(stream), infos)
        return s, infos

    def pcg_block_jacobi(self, M, b, x, tol=1e-10, maxit=10000, fmt="csr", stream=None):
        """CG preconditioned by M, a BlockJacobi built from this matrix."""
        return binding.gko_pcg_block_jacobi(self.handle, _fmt(fmt), M.handle, _dev_f64(b, self.n_rows, "b"),
                                            _dev_f64(x, self.n_rows, "x"), tol, maxit, _stream(stream))

    def bicgstab(self, b, x, tol=1e-10, maxit=10000, fmt="csr", stream=None):
        return binding.gko_bicgstab(self.handle, _fmt(fmt), _dev_f64(b, self.n_rows, "b"),
                                    _dev_f64(x, self.n_rows, "x"), tol, maxit, _stream(stream))

    def gmres(self, b, x, tol=1e-10, restart=30, maxit=10000, fmt="csr", stream=None):
        return binding.gko_gmres(self.handle, _fmt(fmt), _dev_f64(b, self.n_rows, "b"),
                                 _dev_f64(x, self.n_rows, "x"), tol, restart, maxit, _stream(stream))

    def cg_mixed(self, b, x, inner="fp32", tol=1e-10, maxit_outer=50, inner_tol=None, inner_maxit=100000,
                 stream=None, precond="none"):
        """inner_tol None: 1e-2 for FP32 storage, 1e-1 for BF16 (the fastest
        settings measured on a 160^3 variable-coefficient diffusion operator).
        precond "jacobi": the inner solve preconditioned by diag(A_lo)."""
        dt = binding.BF16 if inner == "bf16" else binding.F32
        if inner_tol is None:
            inner_tol = 1e-1 if inner == "bf16" else 1e-2
        if precond == "jacobi":
            return binding.gko_cg_mixed_precond(self.handle, dt, binding.PRECOND_JACOBI, _dev_f64(b, self.n_rows, "b"),
                                                _dev_f64(x, self.n_rows, "x"), tol, maxit_outer, inner_tol,
                                                inner_maxit, _stream(stream))
        return binding.gko_cg_mixed(self.handle, dt, _dev_f64(b, self.n_rows, "b"), _dev_f64(x, self.n_rows, "x"),
                                    tol, maxit_outer, inner_tol, inner_maxit, _stream(stream))

    def features(self, stream=None):
        out = np.zeros(12)
        binding.gko_features(self.handle, out.ctypes.data, _stream(stream))
        return out

    def select_format(self, stream=None):
        return binding.gko_select_format(self.handle, _stream(stream))

    def autotune(self, stream=None):
        """(fmt, config, times_us) of the exhaustive autotuner over the
        candidates this handle can run (times in the order of
        binding.N_CANDIDATES; NaN: not applicable)."""
        return binding.gko_autotune_format(self.handle, _stream(stream))


class BlockJacobi:
    """Owning wrapper of a gko_block_jacobi preconditioner built from a Matrix."""

    def __init__(self, A, max_block_size=8, stream=None):
        self.n_rows = A.n_rows
        self.max_block_size = int(max_block_size)
        self.handle = None
        self.handle = binding.gko_block_jacobi_create(A.handle, self.max_block_size, _stream(stream))

    def close(self):
        if self.handle:
            binding.gko_block_jacobi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self, stream=None):
        """(block_ptr int32 [n_blocks + 1], inv float64 [n_rows * max_block_size]) on the host."""
        nb = binding.gko_block_jacobi_export(self.handle, None, None, _stream(stream))
        bp = np.zeros(nb + 1, dtype=np.int32)
        inv = np.zeros(self.n_rows * self.max_block_size, dtype=np.float64)
        binding.gko_block_jacobi_export(self.handle, bp.ctypes.data, inv.ctypes.data if inv.size else None,
                                        _stream(stream))
        return bp, inv

    def apply(self, r, z, stream=None):
        binding.gko_block_jacobi_apply(self.handle, _dev_f64(r, self.n_rows, "r"), _dev_f64(z, self.n_rows, "z"),
                                       _stream(stream))


class Batch:
    """Owning wrapper of a gko_batch (see synthetic.batched_spd for the layout)."""

    def __init__(self, B, stream=None):
        ro = np.ascontiguousarray(B["row_off"], dtype=np.int64)
        rp = np.ascontiguousarray(B["row_ptr"], dtype=np.int32)
        ci = np.ascontiguousarray(B["col_idx"], dtype=np.int32)
        v = np.ascontiguousarray(B["val"], dtype=np.float64)
        self.count = len(ro) - 1
        self.n_rows = int(ro[-1])
        self.handle = None
        self.handle = binding.gko_batch_create(self.count, ro.ctypes.data, rp.ctypes.data, ci.ctypes.data,
                                               v.ctypes.data, False, _stream(stream))

    def close(self):
        if self.handle:
            binding.gko_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cg(self, b, x, tol=1e-10, maxit=1000, block_size=0, stream=None, with_info=True):
        infos = (SolveInfo * self.count)() if with_info else None
        s = binding.gko_cg_batched(self.handle, _dev_f64(b, self.n_rows, "b"), _dev_f64(x, self.n_rows, "x"), tol,
                                   maxit, block_size, _stream(stream), infos)
        return s, infos

    def autotune(self, b, x, tol=1e-10, maxit=1000, stream=None):
        return binding.gko_batch_autotune(self.handle, _dev_f64(b, self.n_rows, "b"), _dev_f64(x, self.n_rows, "x"),
                                          tol, maxit, _stream(stream))
