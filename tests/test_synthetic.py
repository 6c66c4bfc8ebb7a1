"""Seeded input generators: the published SplitMix64 sequence, determinism,
and the closed-form sizes and structure of every workload."""
import numpy as np
import pytest

import synthetic as syn


def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0: state advances by GAMMA, output = mix64(state)
    # (Steele, Lea, Flood 2014; the reference sequence of Vigna's splitmix64.c)
    st = np.array([1, 2, 3], dtype=np.uint64) * syn.GAMMA
    out = syn.mix64(st)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_draws_are_pure_functions_of_the_counter():
    a = syn.uniform01(7, syn.S_VAL, np.arange(1000, dtype=np.uint64))
    b = syn.uniform01(7, syn.S_VAL, np.arange(500, 1000, dtype=np.uint64))
    assert np.array_equal(a[500:], b)
    assert np.all((a >= 0) & (a < 1))
    c = syn.uniform01(8, syn.S_VAL, np.arange(1000, dtype=np.uint64))
    assert not np.array_equal(a, c)
    k = syn.uniform_int(1, 2, np.arange(100000, dtype=np.uint64), 3, 9)
    assert k.min() == 3 and k.max() == 9


def _check_csr(A):
    rp, ci = A["row_ptr"], A["col_idx"]
    assert rp.dtype == np.int32 and ci.dtype == np.int32 and A["val"].dtype == np.float64
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(ci)
    assert np.all((ci >= 0) & (ci < A["n_cols"]))
    rows = np.repeat(np.arange(A["n_rows"]), np.diff(rp))
    assert np.all((np.diff(ci) > 0) | (np.diff(rows) > 0))  # strictly ascending per row


def test_laplace2d_sizes():
    A = syn.laplace2d(128)
    _check_csr(A)
    assert A["n_rows"] == 16384 and A["row_ptr"][-1] == 81408


def test_stencil27_closed_form_nnz():
    for nx in (1, 2, 5, 17):
        A = syn.stencil27(nx, seed=2)
        _check_csr(A)
        assert A["row_ptr"][-1] == (3 * nx - 2) ** 3
    # the full-size value
    assert (3 * 128 - 2) ** 3 == 55_742_968


def test_diffusion7_structure():
    nx = 9
    A = syn.diffusion7(nx, 1.0, seed=6)
    _check_csr(A)
    n = nx ** 3
    assert A["row_ptr"][-1] == 7 * n - 6 * nx * nx
    assert 7 * 160 ** 3 - 6 * 160 ** 2 == 28_518_400
    D = np.zeros((n, n))
    for i in range(n):
        for k in range(A["row_ptr"][i], A["row_ptr"][i + 1]):
            D[i, A["col_idx"][k]] = A["val"][k]
    assert np.array_equal(D, D.T)
    off = D - np.diag(np.diag(D))
    assert np.all(off <= 0)
    # diagonal dominance: boundary cells strictly, interior cells exactly
    assert np.all(np.diag(D) >= -off.sum(axis=1) - 1e-12)
    assert np.all(np.linalg.eigvalsh(D) > 0)


def test_banded_structure():
    A = syn.banded(3000, 64, 16, seed=3)
    _check_csr(A)
    L = np.diff(A["row_ptr"])
    assert np.all(L == 16)
    rows = np.repeat(np.arange(3000), L)
    assert np.abs(A["col_idx"] - rows).max() <= 64
    assert np.sum(A["col_idx"] == rows) == 3000


def test_powerlaw_mean_and_cap():
    A = syn.powerlaw(200_000, 20.0, 1.5, 20000, seed=4)
    _check_csr(A)
    L = np.diff(A["row_ptr"])
    assert abs(L.mean() - 20.0) <= 0.1
    assert L.max() <= 20000 and L.min() >= 1
    assert 5.0 < A["x_m"] < 9.0


def test_block_diagonal():
    A = syn.block_diagonal(64, 8, seed=5)
    _check_csr(A)
    rows = np.repeat(np.arange(64), 8)
    assert np.all(A["col_idx"] // 8 == rows // 8)


def test_batched_spd_structure():
    B = syn.batched_spd(40, seed=7)
    _check_csr(dict(B, n_cols=B["n_rows"], col_idx=B["col_idx"]) | {"n_cols": 1 << 30})
    assert np.all((B["sizes"] >= 32) & (B["sizes"] <= 1024))
    assert np.all((B["ks"] >= 5) & (B["ks"] <= 15))
    for s in range(40):
        r0, r1 = B["row_off"][s], B["row_off"][s + 1]
        n = r1 - r0
        k0 = B["row_ptr"][r0]
        D = np.zeros((n, n))
        for i in range(n):
            for k in range(B["row_ptr"][r0 + i], B["row_ptr"][r0 + i + 1]):
                D[i, B["col_idx"][k]] = B["val"][k]
        assert np.array_equal(D, D.T)
        off = np.abs(D - np.diag(np.diag(D))).sum(axis=1)
        assert np.allclose(np.diag(D), 1.0 + off, rtol=1e-15, atol=0)
        assert B["nnz_off"][s] == k0


def test_random_csr_edge_cases():
    A = syn.random_csr(50, 0, 5, seed=1)
    assert A["row_ptr"][-1] == 0
    A = syn.random_csr(0, 10, 5, seed=1)
    assert A["n_rows"] == 0 and len(A["row_ptr"]) == 1
    A = syn.random_csr(100, 3, 10, seed=2)
    _check_csr(A)
    assert np.diff(A["row_ptr"]).max() <= 3


@pytest.mark.parametrize("name", ["laplace2d_128", "blockdiag_1M"])
def test_workloads_deterministic(name):
    a, b = syn.workload(name), syn.workload(name)
    assert a["val"].tobytes() == b["val"].tobytes()
    assert a["col_idx"].tobytes() == b["col_idx"].tobytes()


def test_distinct_columns_are_the_first_distinct_draws():
    """Each row's columns are the first L distinct values of its candidate
    sequence (counter = row * 2^32 + j): brute force, one draw at a time, on
    rows that need almost every column of their window (the case the
    generator finishes row by row) and on ordinary rows."""
    n_rows, lo, hi = 40, 0, 299
    lengths = np.array([300 if i % 7 == 0 else (290 if i % 5 == 0 else 3 + i % 11) for i in range(n_rows)])
    rows, cols = syn._distinct_per_row(n_rows, lengths, 9, syn.S_COL, lo, hi)
    for i in range(n_rows):
        got = cols[rows == i]
        want, j = [], 0
        while len(want) < lengths[i]:
            c = int(syn.uniform_int(9, syn.S_COL, np.array([i * (1 << 32) + j], dtype=np.uint64), lo, hi)[0])
            if c not in want:
                want.append(c)
            j += 1
        assert np.array_equal(got, np.sort(want)), i

