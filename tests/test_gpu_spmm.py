"""Multi-RHS SpMM on the GPU against the oracle: every entry of Y within
1e-12 of the compensated reference scale (|alpha| |A| |X| + |beta| |Y|),
bit-exact on integer data."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


MATS = {
    "ragged": lambda: syn.random_csr(1001, 997, 40, seed=2, empty_frac=0.3),
    "powerlaw": lambda: syn.powerlaw(30000, 20.0, 1.5, 5000, seed=5),
    "stencil": lambda: syn.stencil27(16, seed=6),
    "all_empty": lambda: syn.random_csr(100, 90, 0, seed=9),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("k", [1, 3, 8, 17, 40])
def test_spmm_matches_oracle(gko, dev, orc, name, k):
    A = MATS[name]()
    n, m = A["n_rows"], A["n_cols"]
    rng = np.random.default_rng(k)
    X = rng.uniform(-1, 1, size=(m, k))
    Y0 = rng.uniform(-1, 1, size=(n, k))
    for alpha, beta in ((1.0, 0.0), (-0.5, 2.0)):
        ref = orc.spmm_csr(A, X, alpha, beta, Y0)
        Aa = dict(A)
        Aa["val"] = np.abs(A["val"])
        mag = orc.spmm_csr(Aa, np.abs(X), abs(alpha), abs(beta), np.abs(Y0))
        M = gko.Matrix(A)
        Yd = _t(Y0, dev)
        M.spmm(_t(X, dev), Yd, alpha, beta)
        Y = Yd.cpu().numpy()
        assert np.all(np.abs(Y - ref) <= 1e-12 * mag + 1e-300), (name, k, alpha, beta)


def test_spmm_exact_and_beta_zero(gko, dev, orc):
    A = syn.random_csr(3000, 2500, 12, seed=53)
    rng = np.random.default_rng(54)
    A["val"] = rng.integers(-4, 5, size=len(A["val"])).astype(np.float64)
    X = rng.integers(-4, 5, size=(2500, 5)).astype(np.float64)
    M = gko.Matrix(A)
    Yd = _t(np.full((3000, 5), np.nan), dev)  # beta = 0: Y is not read
    M.spmm(_t(X, dev), Yd)
    assert np.array_equal(Yd.cpu().numpy(), orc.spmm_csr(A, X))
    # every column equals the SpMV of that column
    import torch
    for c in range(5):
        y = torch.empty(3000, dtype=torch.float64, device=dev)
        M.spmv(_t(X[:, c], dev), y)
        assert np.array_equal(y.cpu().numpy(), Yd.cpu().numpy()[:, c])
