"""Host-side logic on the CPU: the replica aggregation of the benchmark
across two gloo ranks, the benchmark's byte model, and the selector's
targets, default-kernel rule and regret."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, seconds, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + bench.aggregate_replicas(1e9, seconds[rank], world, "cpu"))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    """Two ranks, 1 GB each in 0.5 s and 0.25 s: both report 2 GB over the
    slower rank's 0.5 s = 4 GB/s."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, (0.5, 0.25), q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gbs, secs in out:
        assert secs == 0.5 and abs(gbs - 4.0) < 1e-12, (rank, gbs, secs)


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate_replicas(3e9, 1.5, 1, "cpu") == (2.0, 1.5)


def test_spmv_byte_model():
    """values + indices + x + y, padding included (β = 0)."""
    import bench
    n, m, nnz = 1000, 900, 5000
    assert bench.spmv_bytes("csr", None, n, m, nnz) == 12 * nnz + 4 * (n + 1) + 8 * m + 8 * n
    assert bench.spmv_bytes("coo", None, n, m, nnz) == 16 * nnz + 8 * m + 8 * n
    ell = [1, n, m, nnz, 7, 1024, 7 * 1024, 0]
    assert bench.spmv_bytes("ell", ell, n, m, nnz) == 12 * 7 * 1024 + 8 * m + 8 * n
    sellp = [1, n, m, nnz, 64, 16, 6000, 1]
    assert bench.spmv_bytes("sellp", sellp, n, m, nnz) == 12 * 6000 + 4 * (2 * 16 + 1) + 8 * m + 8 * n
    hyb = [1, n, m, nnz, 4, 1024, 900, 0]
    assert bench.spmv_bytes("hybrid", hyb, n, m, nnz) == 12 * 4 * 1024 + 16 * 900 + 8 * m + 8 * n


def test_byte_model_matches_the_papers_bound():
    """The marginal bytes of one more stored entry in the benchmark's byte
    model are the per-entry bytes the paper prints for COO and CSR (Sec. 6.1,
    fixture tests/golden/spmv_byte_bound.txt), so its flops per byte are the
    paper's bandwidth / 8 and bandwidth / 6."""
    import bench
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "spmv_byte_bound.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert {r[0] for r in rows} == {"coo", "csr"}
    n, m, nnz = 5000, 5000, 10 ** 6
    for fmt, per_entry, flops_per_byte in rows:
        step = bench.spmv_bytes(fmt, None, n, m, nnz + 1) - bench.spmv_bytes(fmt, None, n, m, nnz)
        assert step == int(per_entry)
        assert 2.0 / step == pytest.approx(float(flops_per_byte), rel=1e-15)


def test_dominant_kernel_roofline():
    """The roofline names the kernel with the largest share of the step:
    launches of one kernel on different matrices are pooled, a hybrid
    without COO part counts as the ELL kernel, and achieved is bytes per
    launch over the mean launch time."""
    import bench
    fam = bench.kernel_family
    assert fam("hybrid", "a", 0) == "ell" and fam("hybrid", "a", 5) == "hybrid"
    assert fam("csr", "a", 9) == "csr:a" and fam("coo", "a", 9) == "coo"
    cases = [dict(matrix="a", fmt="coo", bytes=4e8), dict(matrix="b", fmt="coo", bytes=2e8),
             dict(matrix="b", fmt="hybrid", bytes=3e8), dict(matrix="a", fmt="ell", bytes=3e8),
             dict(matrix="a", fmt="hybrid", bytes=3e8)]
    coo_part = {("b", "hybrid"): 7, ("a", "hybrid"): 0}
    for c in cases:
        c["family"] = fam(c["fmt"], c["matrix"], coo_part.get((c["matrix"], c["fmt"]), 1))
    # the single slowest case is the hybrid (0.5 ms), the busiest kernel is COO (0.4 + 0.3 ms)
    sec = {("a", "coo"): [4e-4, 4e-4], ("b", "coo"): [3e-4, 3e-4], ("b", "hybrid"): [5e-4, 5e-4],
           ("a", "ell"): [1e-4, 1e-4], ("a", "hybrid"): [1e-4, 1e-4]}
    traffic = {"a/coo": 4.4e8, "b/coo": 2.2e8}
    r = bench.dominant_roofline(cases, sec, traffic, 6000.0, "measured")
    assert r["cases"] == ["a/coo", "b/coo"]
    assert r["bytes_per_launch"] == 3e8
    assert r["achieved"] == pytest.approx(3e8 / 3.5e-4 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, rel=1e-3)
    assert r["traffic"] == pytest.approx(3.3e8)
    assert r["share_of_step"] == pytest.approx(14e-4 / 28e-4)
    assert r["slowest_case"]["case"] == "b/hybrid"
    # a kernel whose launches were not all captured has no traffic
    r = bench.dominant_roofline(cases, sec, {"a/coo": 4.4e8}, 6000.0, "measured")
    assert r["traffic"] is None
    # the ELL kernel (plain ELL and the hybrid without COO part) takes over when it dominates
    sec[("a", "ell")] = [9e-4, 9e-4]
    r = bench.dominant_roofline(cases, sec, traffic, 6000.0, "measured")
    assert r["cases"] == ["a/ell", "a/hybrid"] and r["kernel"] == "ell_kernel"


def test_launch_count_model():
    """One launch per SpMV, plus the fix-up of the equal-nnz kernel once the
    entries span more than one tile of 64 x 11."""
    import bench
    assert bench.kernel_launches("coo", 704) == 1 and bench.kernel_launches("coo", 705) == 2
    assert bench.kernel_launches("hybrid", 0) == 1 and bench.kernel_launches("hybrid", 10 ** 6) == 3
    assert bench.kernel_launches("csr", 10 ** 6) == 1 and bench.kernel_launches("ell", 10 ** 6) == 1


def test_selector_targets_regret_and_default_rule(gko):
    from paper_2011_08879_gb300 import selector as sel
    from paper_2011_08879_gb300 import binding as B
    T = np.array([2e-4, 1e-4, np.nan, 1e-1] + [np.nan] * (len(sel.CANDIDATES) - 4))
    y, m = sel.targets(T)
    assert m[:4].tolist() == [1, 1, 0, 1] and m[4:].sum() == 0
    assert abs(y[0] - np.log10(2.0)) < 1e-6 and y[1] == 0.0
    assert y[3] == sel.TARGET_CAP  # 1000x slower, capped
    TT = np.array([[1.0, 2.0, np.nan], [4.0, 1.0, 3.0]])
    r = sel.regret(TT, np.array([1, 2]))
    assert np.allclose(r, [1.0, 2.0])
    r = sel.regret(TT, np.array([2, 1]))  # an unmeasured choice counts as the worst measured time
    assert np.allclose(r, [1.0, 0.0])
    names = sel.CLASS_NAMES
    F = np.zeros((4, 12))
    F[:, 2] = [7.0, 16.0, 27.0, 20.0]   # mean row length
    F[:, 4] = [7.0, 16.0, 27.0, 20000]  # max row length
    got = [names[c] for c in sel.default_csr_class(F)]
    want = ["csr/%d" % c for c in (B.CFG_CSR_SUBWARP_1, B.CFG_CSR_ROWBLOCK, B.CFG_CSR_SUBWARP_4, B.CFG_CSR_BINNED)]
    assert got == want


def test_traffic_scaled_from_the_small_capture(tmp_path):
    """DRAM traffic per launch is the captured ratio (DRAM over algorithmic
    bytes on the quarter-size matrix of the same kind) times the full case's
    algorithmic bytes, and is withheld when the capture was taken on other
    kernel sources."""
    import bench
    f = tmp_path / "traffic.txt"
    cases = [dict(matrix="stencil27_128", fmt="coo", bytes=925.4e6), dict(matrix="banded_4M", fmt="ell", bytes=1e9)]
    f.write_text("source %s\nratio stencil27/coo 1.002\n" % bench.kernel_source_hash())
    t = bench.profile_traffic(cases, str(f))
    assert t == {"stencil27_128/coo": 1.002 * 925.4e6}
    f.write_text("source 0000\nratio stencil27/coo 1.002\n")
    assert bench.profile_traffic(cases, str(f)) == {}
