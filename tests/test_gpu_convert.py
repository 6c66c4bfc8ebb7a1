"""Format conversions on the device against the oracle: bit-exact in every
index and value array (padding included), and round trips CSR -> X -> CSR
identical to the input."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def cases():
    A = syn.random_csr(777, 900, 30, seed=40, empty_frac=0.25)
    A["val"] = A["val"].copy()
    A["val"][::5] = 0.0
    A["val"][1::9] = -0.0  # signed zeros must survive bit for bit
    return {
        "ragged": A,
        "powerlaw": syn.powerlaw(40000, 20.0, 1.5, 4000, seed=41),
        "stencil": syn.stencil27(17, seed=42),
        "diffusion": syn.diffusion7(12, seed=43),
        "one_row": syn.random_csr(1, 64, 64, seed=44),
        "all_empty": syn.random_csr(70, 70, 0, seed=45),
    }


def same(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return a.dtype == b.dtype and a.shape == b.shape and a.tobytes() == b.tobytes()


@pytest.mark.parametrize("name", list(cases()))
def test_conversions_bit_exact(gko, dev, orc, name):
    A = cases()[name]
    n, m = A["n_rows"], A["n_cols"]
    M = gko.Matrix(A)
    M.convert("coo")
    g = M.export("coo")
    o = orc.to_coo(A)
    assert same(g["row"], o["row"]) and same(g["col"], o["col"]) and same(g["val"], o["val"])

    if orc.max_row_len(A) * orc.ell_n_pad(n) <= max(4 * len(A["val"]), 1 << 22):
        M.convert("ell")
        g = M.export("ell")
        o = orc.to_ell(A)
        assert g["info"][4] == o["K"] and g["info"][5] == o["n_pad"]
        assert same(g["col"], o["col"]) and same(g["val"], o["val"])

    M.set_params(ell_factor=1e6)  # conversions are checked whatever the padding
    for S, f in ((64, 1), (32, 1), (32, 4), (8, 2)):
        M.set_params(sellp_slice=S, sellp_stride=f)
        M.convert("sellp")
        g = M.export("sellp")
        o = orc.to_sellp(A, S, f)
        assert same(g["slice_len"], o["slice_len"]) and same(g["slice_set"], o["slice_set"])
        assert same(g["col"], o["col"]) and same(g["val"], o["val"])

    M.convert("hybrid")
    g = M.export("hybrid")
    o = orc.to_hybrid(A)
    assert g["info"][4] == o["K"]
    for k in ("ell_col", "ell_val", "coo_row", "coo_col", "coo_val"):
        assert same(g[k], o[k]), k


@pytest.mark.parametrize("name", list(cases()))
def test_round_trips(gko, dev, name):
    A = cases()[name]
    for f in ("coo", "ell", "sellp", "hybrid"):
        M = gko.Matrix(A)
        try:
            M.convert(f)
        except gko.GkoError as e:
            assert f in ("ell", "sellp") and e.status == gko.binding.ERR_FORMAT_TOO_LARGE
            continue
        M.release("csr")
        assert not M.has("csr")
        M.convert("csr", src=f)
        g = M.export("csr")
        assert same(g["row_ptr"], A["row_ptr"]), f
        assert same(g["col"], A["col_idx"]), f
        assert same(g["val"], A["val"]), f


def test_full_size_conversions_bit_exact(gko, dev, orc):
    """Power-law at full size (2M rows, 20k-long rows): SELL-P and hybrid
    against the oracle; COO by its definition."""
    A = syn.workload("powerlaw_2M")
    M = gko.Matrix(A)
    M.convert("hybrid")
    g = M.export("hybrid")
    o = orc.to_hybrid(A)
    for k in ("ell_col", "ell_val", "coo_row", "coo_col", "coo_val"):
        assert same(g[k], o[k]), k
    with pytest.raises(gko.GkoError) as e:  # 13.9x padding: over the limit
        M.convert("sellp")
    assert e.value.status == gko.binding.ERR_FORMAT_TOO_LARGE
    M.convert("coo")
    g = M.export("coo")
    assert same(g["row"], np.repeat(np.arange(A["n_rows"], dtype=np.int32), np.diff(A["row_ptr"])))
    B = syn.workload("banded_4M")
    MB = gko.Matrix(B)
    MB.convert("sellp")
    g = MB.export("sellp")
    o = orc.to_sellp(B, 64, 1)
    for k in ("slice_len", "slice_set", "col", "val"):
        assert same(g[k], o[k]), k
    MB.convert("ell")
    g = MB.export("ell")
    o = orc.to_ell(B)
    assert same(g["col"], o["col"]) and same(g["val"], o["val"])
