"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

This module only *draws* inputs: sparsity patterns, matrix values, right-hand
sides and vectors.  It holds none of the arithmetic the library computes
(no products, no sums over a row, no solver step, no format conversion), so
the oracle and the CUDA path can both take their inputs from here without
sharing any of the method's code.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
2014): the i-th draw of stream ``key`` is ``mix64(key + (i + 1) * GAMMA)``
where ``mix64`` is the SplitMix64 finaliser.  A uniform double in [0, 1) is
``(h >> 11) * 2**-53``.  Every array is a pure function of (seed, stream,
index), so any entry can be regenerated on its own.

All matrices are returned in CSR with int32 indices, float64 values and
column indices sorted ascending inside each row, as a dict with keys
``n_rows, n_cols, row_ptr, col_idx, val`` (plus generator-specific extras).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53 = float(2.0 ** -53)

# Stream identifiers: one independent SplitMix64 stream per purpose.
S_VAL, S_COL, S_LEN, S_X, S_B, S_KAPPA, S_SIZE, S_PART, S_STRUCT = range(1, 10)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of stream ``stream`` under ``seed``: one SplitMix64 draw of the pair."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(stream)
    return np.uint64(mix64(np.array([s], dtype=np.uint64))[0])


def draw_u64(seed: int, stream: int, idx) -> np.ndarray:
    """Raw 64-bit draws ``idx`` (uint64 array of counters) of one stream."""
    key = stream_key(seed, stream)
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + (idx + np.uint64(1)) * GAMMA)


def uniform01(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (draw_u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * _TWO53


def uniform_pm1(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform doubles in [-1, 1): 2u - 1."""
    return 2.0 * uniform01(seed, stream, idx) - 1.0


def uniform_int(seed: int, stream: int, idx, lo, hi) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive; lo/hi may be arrays): lo + floor(u*(hi-lo+1))."""
    u = uniform01(seed, stream, idx)
    lo = np.asarray(lo, dtype=np.int64)
    span = np.asarray(hi, dtype=np.int64) - lo + 1
    return lo + np.minimum((u * span).astype(np.int64), span - 1)


def vector(n: int, seed: int, stream: int = S_X) -> np.ndarray:
    """A length-n float64 vector uniform in [-1, 1)."""
    return uniform_pm1(seed, stream, np.arange(n, dtype=np.uint64))


def _csr_from_sorted(n_rows, n_cols, rows, cols, val=None, seed=None, **extra):
    """Pack (row, col) pairs already sorted by (row, col) into CSR.

    If ``val`` is None the values are drawn uniform in [-1, 1) indexed by the
    entry's CSR position.
    """
    counts = np.bincount(rows, minlength=n_rows) if len(rows) else np.zeros(n_rows, np.int64)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32 indices")
    if val is None:
        val = uniform_pm1(seed, S_VAL, np.arange(len(cols), dtype=np.uint64))
    d = dict(n_rows=int(n_rows), n_cols=int(n_cols), row_ptr=row_ptr.astype(np.int32),
             col_idx=np.asarray(cols, dtype=np.int32), val=np.asarray(val, dtype=np.float64))
    d.update(extra)
    return d


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """Sorted distinct values of an integer array (sort-based)."""
    a = np.sort(a)
    if a.size:
        a = a[np.concatenate(([True], a[1:] != a[:-1]))]
    return a


_TAIL_ROWS = 256  # rows left when _distinct_per_row switches to finishing them one at a time


def _finish_rows(active, need, next_j, seen_all, stride, seed, stream, lo, hi, exclude):
    """Keys completing each row of ``active``: its next ``need[i]`` distinct
    values of the candidate sequence (from position next_j[i] on, skipping
    the excluded value and the row's values in ``seen_all``), in sequence
    order.  Drawing a longer run and keeping the first new values in order
    gives the same values as drawing the deficit batch by batch."""
    out = []
    for i in active:
        lo_i, hi_i = int(lo[i]), int(hi[i])
        a, b = np.searchsorted(seen_all, [i * stride, (i + 1) * stride])
        seen = seen_all[a:b] - i * stride  # offsets the row already has (sorted)
        left, j = int(need[i]), int(next_j[i])
        while left > 0:
            chunk = max(4 * left, 1024)
            counter = np.uint64(i) * np.uint64(1 << 32) + np.arange(j, j + chunk, dtype=np.uint64)
            c = uniform_int(seed, stream, counter, lo_i, hi_i)
            if exclude is not None:
                c = c[c != exclude[i]]
            vals, first = np.unique(c - lo_i, return_index=True)
            vals = vals[np.argsort(first, kind="stable")]  # distinct values in order of first draw
            vals = vals[~np.isin(vals, seen)]
            take = vals[:left]
            out.append(i * stride + take)
            seen = np.union1d(seen, take)
            left -= take.size
            j += chunk
    return _sorted_unique(np.concatenate(out)) if out else np.zeros(0, dtype=np.int64)


def _distinct_per_row(n_rows, lengths, seed, stream, lo, hi, exclude=None):
    """For each row i, the first ``lengths[i]`` distinct integers of the row's
    candidate sequence c_{i,j} = uniform_int(counter = i * 2**32 + j, lo_i, hi_i),
    j = 0, 1, 2, ..., skipping ``exclude[i]`` when given.

    Returns (rows, cols) sorted by (row, col).  Drawing in batches of the
    remaining deficit gives the same set as drawing one candidate at a time,
    because a batch of d draws adds at most d new values.
    """
    lengths = np.asarray(lengths, dtype=np.int64)
    lo = np.broadcast_to(np.asarray(lo, dtype=np.int64), (n_rows,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.int64), (n_rows,))
    width = int(np.max(hi - lo + 1)) if n_rows else 1
    stride = np.int64(max(width, 1))
    need = lengths.copy()
    next_j = np.zeros(n_rows, dtype=np.int64)

    def draw(active):
        d = need[active]
        r = np.repeat(active, d)
        starts = np.repeat(next_j[active], d)
        j = starts + np.arange(r.size, dtype=np.int64) - np.repeat(np.cumsum(d) - d, d)
        counter = r.astype(np.uint64) * np.uint64(1 << 32) + j.astype(np.uint64)
        c = uniform_int(seed, stream, counter, lo[r], hi[r])
        keep = np.ones(c.size, dtype=bool) if exclude is None else (c != exclude[r])
        next_j[active] += d
        # key = (row, column offset inside the row's window): unique per entry
        return _sorted_unique(r[keep] * stride + (c[keep] - lo[r[keep]]))

    base = draw(np.arange(n_rows, dtype=np.int64))  # sorted, distinct
    need -= np.bincount(base // stride, minlength=n_rows)
    extra = np.zeros(0, dtype=np.int64)  # sorted keys added by later rounds
    while True:
        active = np.nonzero(need > 0)[0]
        if active.size == 0:
            break
        if active.size <= _TAIL_ROWS:
            # few rows left (typically long rows collecting their last
            # columns): finish them row by row, see _finish_rows
            seen_all = _sorted_unique(np.concatenate([base, extra])) if extra.size else base
            extra = np.concatenate([extra, _finish_rows(active, need, next_j, seen_all, stride, seed, stream,
                                                        lo, hi, exclude)])
            break
        keys = draw(active)
        for seen in (base, extra):
            if seen.size and keys.size:
                pos = np.minimum(np.searchsorted(seen, keys), seen.size - 1)
                keys = keys[seen[pos] != keys]
        extra = _sorted_unique(np.concatenate([extra, keys]))
        need -= np.bincount(keys // stride, minlength=n_rows)
    keys = _sorted_unique(np.concatenate([base, extra])) if extra.size else base
    rows = keys // stride
    cols = lo[rows] + keys % stride
    return rows, cols


def laplace2d(nx: int = 128) -> dict:
    """2D 5-point Laplacian on an nx x nx grid: diagonal 4, neighbours -1,
    Dirichlet boundary (out-of-grid neighbours dropped), row index i + nx*j."""
    n = nx * nx
    idx = np.arange(n, dtype=np.int64)
    i, j = idx % nx, idx // nx
    parts = []
    for dj, di, v in ((-1, 0, -1.0), (0, -1, -1.0), (0, 0, 4.0), (0, 1, -1.0), (1, 0, -1.0)):
        ok = (i + di >= 0) & (i + di < nx) & (j + dj >= 0) & (j + dj < nx)
        parts.append((idx[ok], idx[ok] + di + nx * dj, np.full(int(ok.sum()), v)))
    rows = np.concatenate([p[0] for p in parts])
    cols = np.concatenate([p[1] for p in parts])
    vals = np.concatenate([p[2] for p in parts])
    order = np.lexsort((cols, rows))
    return _csr_from_sorted(n, n, rows[order], cols[order], vals[order], grid=(nx, nx))


def convdiff2d(nx: int = 64, wind: float = 0.5) -> dict:
    """Nonsymmetric 2D convection-diffusion operator on an nx x nx grid: the
    5-point Laplacian (diagonal 4, neighbours -1, Dirichlet, row i + nx*j)
    plus a centred first difference along i with weight `wind` (east
    neighbour -1 + wind/2, west neighbour -1 - wind/2)."""
    A = laplace2d(nx)
    n = A["n_rows"]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A["row_ptr"]))
    d = A["col_idx"].astype(np.int64) - rows
    v = A["val"].copy()
    v[d == 1] += 0.5 * wind
    v[d == -1] -= 0.5 * wind
    A["val"] = v
    return A


def stencil27(nx: int = 128, seed: int = 2) -> dict:
    """3D 27-point stencil pattern on an nx^3 grid (row i + nx*j + nx^2*k),
    out-of-grid neighbours dropped, values uniform in [-1, 1)."""
    n = nx ** 3
    idx = np.arange(n, dtype=np.int64)
    i, j, k = idx % nx, (idx // nx) % nx, idx // (nx * nx)
    cols = np.empty((27, n), dtype=np.int64)
    ok = np.empty((27, n), dtype=bool)
    t = 0
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                ok[t] = ((i + di >= 0) & (i + di < nx) & (j + dj >= 0) & (j + dj < nx)
                         & (k + dk >= 0) & (k + dk < nx))
                cols[t] = idx + di + nx * dj + nx * nx * dk
                t += 1
    okT = ok.T
    c = cols.T[okT]
    r = np.broadcast_to(idx[:, None], (n, 27))[okT]
    del cols, ok, okT
    return _csr_from_sorted(n, n, r, c, seed=seed)


def banded(n: int = 4_000_000, half_bw: int = 64, per_row: int = 16, seed: int = 3) -> dict:
    """Random banded matrix: each row holds its diagonal plus per_row-1
    distinct columns drawn uniformly from the clipped window
    [i - half_bw, i + half_bw] (so |i - j| <= half_bw); values uniform [-1, 1)."""
    idx = np.arange(n, dtype=np.int64)
    lo = np.maximum(0, idx - half_bw)
    hi = np.minimum(n - 1, idx + half_bw)
    avail = hi - lo  # window size minus the diagonal
    lengths = np.minimum(per_row - 1, avail)
    r, c = _distinct_per_row(n, lengths, seed, S_COL, lo, hi, exclude=idx)
    key = np.sort(np.concatenate([r * n + c, idx * n + idx]))
    return _csr_from_sorted(n, n, key // n, key % n, seed=seed)


def powerlaw_lengths(n: int, seed: int, mean: float = 20.0, alpha: float = 1.5,
                     max_len: int = 20000) -> tuple[np.ndarray, float]:
    """Row lengths with a Pareto tail: L = min(max_len, floor(x_m * U**(-1/alpha))),
    U in (0, 1], with x_m found by bisection so that sum(L) is within 0.5 % of
    mean * n.  Returns (lengths, x_m)."""
    u = 1.0 - uniform01(seed, S_LEN, np.arange(n, dtype=np.uint64))  # (0, 1]
    base = u ** (-1.0 / alpha)

    def total(xm):
        return float(np.minimum(max_len, np.floor(xm * base)).sum())

    lo, hi = 0.5, float(mean) * 4
    target = mean * n
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < target:
            lo = mid
        else:
            hi = mid
        if abs(total(mid) - target) <= 0.005 * target and hi - lo < 1e-6:
            break
    xm = 0.5 * (lo + hi)
    lengths = np.minimum(max_len, np.floor(xm * base)).astype(np.int64)
    lengths = np.minimum(lengths, n)
    return lengths, xm


def powerlaw(n: int = 2_000_000, mean: float = 20.0, alpha: float = 1.5, max_len: int = 20000,
             seed: int = 4) -> dict:
    """Power-law row lengths (powerlaw_lengths) with distinct columns uniform
    over [0, n), sorted; values uniform in [-1, 1)."""
    lengths, xm = powerlaw_lengths(n, seed, mean, alpha, max_len)
    r, c = _distinct_per_row(n, lengths, seed, S_COL, 0, n - 1)
    return _csr_from_sorted(n, n, r, c, seed=seed, x_m=xm)


def block_diagonal(n: int = 1_000_000, b: int = 8, seed: int = 5) -> dict:
    """Block-diagonal matrix of dense b x b blocks (n/b blocks), values uniform [-1, 1)."""
    if n % b:
        raise ValueError("n must be a multiple of the block size")
    idx = np.arange(n, dtype=np.int64)
    r = np.repeat(idx, b)
    c = (np.repeat(idx // b * b, b) + np.tile(np.arange(b), n))
    return _csr_from_sorted(n, n, r, c, seed=seed)


def uniform_random(n: int, per_row_mean: float, seed: int, n_cols: int | None = None) -> dict:
    """Uniform random pattern: row length uniform in [0, 2*mean] (clipped to
    n_cols), distinct columns uniform over [0, n_cols)."""
    m = n if n_cols is None else n_cols
    hi = max(0, int(round(2 * per_row_mean)))
    lengths = uniform_int(seed, S_LEN, np.arange(n, dtype=np.uint64), 0, hi)
    lengths = np.minimum(lengths, m)
    r, c = _distinct_per_row(n, lengths, seed, S_COL, 0, m - 1)
    return _csr_from_sorted(n, m, r, c, seed=seed)


def random_csr(n_rows: int, n_cols: int, max_per_row: int, seed: int,
               empty_frac: float = 0.0) -> dict:
    """Small irregular test matrices: row lengths uniform in [0, max_per_row]
    (clipped to n_cols), a fraction ``empty_frac`` of rows forced empty."""
    lengths = uniform_int(seed, S_LEN, np.arange(n_rows, dtype=np.uint64), 0, max_per_row)
    lengths = np.minimum(lengths, n_cols)
    if empty_frac > 0:
        e = uniform01(seed, S_STRUCT, np.arange(n_rows, dtype=np.uint64)) < empty_frac
        lengths[e] = 0
    if n_cols == 0:
        lengths[:] = 0
    r, c = _distinct_per_row(n_rows, lengths, seed, S_COL, 0, max(n_cols - 1, 0))
    return _csr_from_sorted(n_rows, n_cols, r, c, seed=seed)


def diffusion7(nx: int = 160, sigma: float = 1.0, seed: int = 6) -> dict:
    """SPD 3D 7-point variable-coefficient diffusion operator on an nx^3 grid.

    Cell coefficients kappa_c = exp(sigma * z_c) with z_c standard normal from
    the Box-Muller transform of two uniforms; the coefficient of the face
    between cells a and b is the harmonic mean 2 k_a k_b / (k_a + k_b); a
    Dirichlet boundary face of cell c contributes 2 k_c.  Off-diagonal
    A_ij = -(face coefficient), A_ii = sum of the cell's six face coefficients.
    """
    n = nx ** 3
    idx = np.arange(n, dtype=np.int64)
    u1 = 1.0 - uniform01(seed, S_KAPPA, 2 * idx.astype(np.uint64))
    u2 = uniform01(seed, S_KAPPA, 2 * idx.astype(np.uint64) + np.uint64(1))
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    kappa = np.exp(sigma * z)
    i, j, k = idx % nx, (idx // nx) % nx, idx // (nx * nx)
    coord = (i, j, k)
    stride = (1, nx, nx * nx)
    diag = np.zeros(n)
    offs = []  # (delta, ok-mask, face coefficient)
    for axis in (2, 1, 0):
        for sgn in (-1, 1):
            ok = (coord[axis] + sgn >= 0) & (coord[axis] + sgn < nx)
            nb = np.where(ok, idx + sgn * stride[axis], idx)
            ka, kb = kappa, kappa[nb]
            face = np.where(ok, 2.0 * ka * kb / (ka + kb), 2.0 * ka)
            diag += face
            offs.append((sgn * stride[axis], ok, face))
    # column order: -z, -y, -x, self, +x, +y, +z  (ascending)
    order = [offs[0], offs[2], offs[4], None, offs[5], offs[3], offs[1]]
    cols, vals, oks = [], [], []
    for o in order:
        if o is None:
            cols.append(idx)
            vals.append(diag)
            oks.append(np.ones(n, dtype=bool))
        else:
            d, ok, face = o
            cols.append(idx + d)
            vals.append(-face)
            oks.append(ok)
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    K = np.stack(oks, axis=1)
    r = np.broadcast_to(idx[:, None], C.shape)[K]
    return _csr_from_sorted(n, n, r, C[K], V[K], kappa=kappa)


def batched_spd(count: int = 4096, seed: int = 7, n_min: int = 32, n_max: int = 1024,
                k_min: int = 5, k_max: int = 15) -> dict:
    """``count`` independent sparse SPD systems of uneven size.

    System s has n_s ~ U{n_min..n_max} rows and k_s ~ U{k_min..k_max}.  Each
    row i draws floor((k_s - 1) / 2) partners j != i uniformly; the pair gets
    a_ij = a_ji ~ U[-1, 1), the first draw of a pair (in row, then draw order)
    fixing its value.  a_ii = 1 + sum_j |a_ij| makes the matrix strictly
    diagonally dominant with a positive diagonal, hence SPD.  The right-hand
    side is uniform in [-1, 1).

    Returned CSR blocks are concatenated: rows of system s are
    [row_off[s], row_off[s+1]) and its column indices are local to the system
    (0..n_s-1); row_ptr is global over the concatenation.
    """
    sid = np.arange(count, dtype=np.uint64)
    ns = uniform_int(seed, S_SIZE, 2 * sid, n_min, n_max)
    ks = uniform_int(seed, S_SIZE, 2 * sid + np.uint64(1), k_min, k_max)
    row_off = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(ns, out=row_off[1:])
    N = int(row_off[-1])
    sys_of_row = np.repeat(np.arange(count, dtype=np.int64), ns)
    local = np.arange(N, dtype=np.int64) - row_off[sys_of_row]
    per = (ks - 1) // 2
    per_row = per[sys_of_row]
    R = np.repeat(np.arange(N, dtype=np.int64), per_row)  # global row of each draw
    t = np.arange(R.size, dtype=np.int64) - np.repeat(np.cumsum(per_row) - per_row, per_row)
    s_of = sys_of_row[R]
    n_of = ns[s_of]
    counter = R.astype(np.uint64) * np.uint64(64) + t.astype(np.uint64)
    j = uniform_int(seed, S_PART, counter, 0, n_of - 2)
    li = local[R]
    j = j + (j >= li)
    v = uniform_pm1(seed, S_VAL, counter)
    a, b = np.minimum(li, j), np.maximum(li, j)
    key = (s_of * 1024 + a) * 1024 + b
    order0 = np.argsort(key, kind="stable")  # stable: equal keys stay in (row, draw) order
    ks_sorted = key[order0]
    first = order0[np.concatenate(([True], ks_sorted[1:] != ks_sorted[:-1]))]
    s_u, a_u, b_u, v_u = s_of[first], a[first], b[first], v[first]
    base = row_off[s_u]
    rows = np.concatenate([base + a_u, base + b_u])
    cols = np.concatenate([b_u, a_u])
    vals = np.concatenate([v_u, v_u])
    absum = np.bincount(rows, weights=np.abs(vals), minlength=N)
    rows = np.concatenate([rows, np.arange(N, dtype=np.int64)])
    cols = np.concatenate([cols, local])
    vals = np.concatenate([vals, 1.0 + absum])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rhs = uniform_pm1(seed, S_B, np.arange(N, dtype=np.uint64))
    d = _csr_from_sorted(N, N, rows, cols, vals, row_off=row_off, sizes=ns, ks=ks, rhs=rhs)
    nnz_off = d["row_ptr"][row_off].astype(np.int64)
    d["nnz_off"] = nnz_off
    return d


SWEEP_STRUCTURES = ("stencil", "banded", "powerlaw", "random")


def sweep_params(seed: int, n_min: float = 1e4, n_max: float = 4e6, m_min: float = 4.0, m_max: float = 200.0,
                 nnz_cap: float = 3e7) -> dict:
    """Shape of one selector-sweep matrix: structure equiprobable over
    SWEEP_STRUCTURES, rows log-uniform in [n_min, n_max], mean entries per
    row log-uniform in [m_min, m_max]; rows are reduced so that rows * mean
    stays below nnz_cap (3e7 entries, 480 MB as COO: the full product of the
    ranges would reach 8e8 entries, beyond what the host generates in the
    time of one sweep)."""
    u = uniform01(seed, S_STRUCT, np.arange(4, dtype=np.uint64))
    structure = SWEEP_STRUCTURES[min(3, int(u[0] * 4))]
    n = 10 ** (math.log10(n_min) + u[1] * (math.log10(n_max) - math.log10(n_min)))
    m = 10 ** (math.log10(m_min) + u[2] * (math.log10(m_max) - math.log10(m_min)))
    n = int(max(n_min / 4, min(n, nnz_cap / m)))
    return dict(structure=structure, n=n, mean=m, u3=float(u[3]))


def sweep_matrix(seed: int, **kw) -> dict:
    """One matrix of the selector sweep (see sweep_params); values uniform
    in [-1, 1)."""
    p = sweep_params(seed, **kw)
    n, m, s = p["n"], p["mean"], p["structure"]
    if s == "stencil":  # 2D 5-point, 3D 7-point or 3D 27-point pattern by u3
        kind = int(p["u3"] * 3)
        if kind == 0:
            side = max(2, int(round(n ** 0.5)))
            A = laplace2d(side)
            A["val"] = uniform_pm1(seed, S_VAL, np.arange(len(A["col_idx"]), dtype=np.uint64))
        elif kind == 1:
            side = max(2, int(round(n ** (1 / 3))))
            A = diffusion7(side, 1.0, seed=seed)
            A["val"] = uniform_pm1(seed, S_VAL, np.arange(len(A["col_idx"]), dtype=np.uint64))
        else:
            A = stencil27(max(2, int(round(n ** (1 / 3)))), seed=seed)
    elif s == "banded":
        per_row = max(2, int(round(m)))
        half_bw = max(per_row, int(round(per_row * (1 + 7 * p["u3"]))))
        A = banded(n, half_bw, per_row, seed=seed)
    elif s == "powerlaw":
        A = powerlaw(n, m, 1.5, min(20000, n), seed=seed)
    else:
        A = uniform_random(n, m, seed)
    A["structure"] = s
    return A


# Workloads of the benchmark configurations, with their seeds.
def workload(name: str) -> dict:
    """The named synthetic workload at full size."""
    if name == "laplace2d_128":
        return laplace2d(128)
    if name == "stencil27_128":
        return stencil27(128, seed=2)
    if name == "banded_4M":
        return banded(4_000_000, 64, 16, seed=3)
    if name == "powerlaw_2M":
        return powerlaw(2_000_000, 20.0, 1.5, 20000, seed=4)
    if name == "blockdiag_1M":
        return block_diagonal(1_000_000, 8, seed=5)
    # quarter-size matrices of the same four kinds (profiling captures)
    if name == "stencil27_80":
        return stencil27(80, seed=2)
    if name == "banded_1M":
        return banded(1_000_000, 64, 16, seed=3)
    if name == "powerlaw_500k":
        return powerlaw(500_000, 20.0, 1.5, 20000, seed=4)
    if name == "blockdiag_250k":
        return block_diagonal(250_000, 8, seed=5)
    if name == "diffusion7_160":
        return diffusion7(160, 1.0, seed=6)
    if name == "batched_4096":
        return batched_spd(4096, seed=7)
    raise KeyError(name)


SPMV_SWEEP = ("stencil27_128", "banded_4M", "powerlaw_2M", "blockdiag_1M")
SPMV_SWEEP_SMALL = ("stencil27_80", "banded_1M", "powerlaw_500k", "blockdiag_250k")
