#!/usr/bin/env python3
"""Benchmark of the sparse hot path on GB300.

One step = one FP64 SpMV (y = A x) in every available format (CSR, COO,
ELL, SELL-P, hybrid) on each matrix of the SpMV sweep: a 27-point stencil on
a 128^3 grid, a random banded matrix (4M rows, bandwidth 64, 16/row), a
power-law matrix (2M rows, Pareto tail 1.5, mean 20/row, max 20k) and a
block-diagonal matrix (1M rows, 8x8 blocks).  L2 is flushed (a 512 MB
write) before every SpMV and only the SpMV kernels are timed, with CUDA
events on the launching stream.  value = algorithmic bytes (values +
indices + x + y) of all SpMVs / their total time.

Extras in the same JSON line: the same metric end to end through
gko_spmv_host (host buffers, copies inside the timed region), the roofline
of the dominant kernel, the oracle timed on the host cores, CG time to a
1e-10 relative residual (5-point Laplacian 128^2; 7-point diffusion 160^3
in FP64 vs FP32/BF16 + FP64 refinement) and batched CG on 4096 systems.

--impl reference times the CPU oracle on the same workload (bounded
sample per step).  Multi-GPU (torchrun): every rank runs its own replica.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

SWEEP = syn.SPMV_SWEEP
FORMATS = ("csr", "coo", "ell", "sellp", "hybrid")
L2_FLUSH_BYTES = 512 << 20
CACHE = os.environ.get("GKO_BENCH_CACHE", "/tmp/gko_gb300_bench_cache")


# ------------------------------------------------------------------ inputs

def load_workload(name):
    """Synthetic workload, cached as .npz between runs of one session."""
    os.makedirs(CACHE, exist_ok=True)
    path = os.path.join(CACHE, name + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return {k: (z[k].item() if z[k].ndim == 0 else z[k]) for k in z.files}
    A = syn.workload(name)
    keep = {k: v for k, v in A.items() if isinstance(v, (np.ndarray, int, float))}
    np.savez(path + ".tmp.npz", **keep)
    os.replace(path + ".tmp.npz", path)
    return A


# ------------------------------------------------------------- byte model

def spmv_bytes(fmt, info, n, m, nnz, s_v=8):
    """Algorithmic bytes of one y = A x (beta = 0: y written once, x read
    once): values + indices + x + y.  Padding slots count (they are moved)."""
    x_y = s_v * m + s_v * n
    if fmt == "csr":
        return (s_v + 4) * nnz + 4 * (n + 1) + x_y
    if fmt == "coo":
        return (s_v + 8) * nnz + x_y
    if fmt == "ell":
        return (s_v + 4) * info[6] + x_y
    if fmt == "sellp":
        return (s_v + 4) * info[6] + 4 * (2 * info[5] + 1) + x_y
    if fmt == "hybrid":
        return (s_v + 4) * info[4] * info[5] + (s_v + 8) * info[6] + x_y
    raise KeyError(fmt)


def csr_default_launches(A):
    """Launches of the default CSR SpMV: one kernel (uniform rows: subwarp
    or row-block kernel; skewed rows: the one-launch binned kernel)."""
    return 1


def kernel_launches(fmt, nnz_or_coo, tile=704, csr_launches=1):
    """Launches of this library per SpMV (load-balanced kernels add a fix-up
    launch when they span more than one tile)."""
    seg = 1 + (1 if nnz_or_coo > tile else 0)
    return {"csr": csr_launches, "coo": seg, "ell": 1, "sellp": 1, "hybrid": 1 + (seg if nnz_or_coo else 0)}[fmt]


def kernel_family(fmt, matrix, coo_part):
    """Kernel that carries a (matrix, format) SpMV: COO, ELL and SELL-P have
    one kernel each; a hybrid without COO part runs the ELL kernel alone;
    the default CSR kernel follows the row lengths (one per sweep matrix)."""
    if fmt == "hybrid" and not coo_part:
        return "ell"
    if fmt == "csr":
        return "csr:" + matrix
    return fmt


FAMILY_LABEL = {
    "coo": "seg_spmv_kernel<11|13> (COO, equal-nnz tiles of 64 threads) + fix-up",
    "ell": "ell_kernel",
    "sellp": "sellp_kernel",
    "hybrid": "ell_kernel + seg_spmv_kernel<11|13> (COO part, accumulate) + fix-up",
}


def dominant_roofline(cases, seconds, traffic, peak, peak_kind):
    """Roofline of the kernel with the largest share of the step's device
    time.  cases: dicts with matrix, fmt, bytes, family; seconds: per case,
    the list of its timed launches; traffic: DRAM bytes per launch by
    'matrix/fmt' (ncu).  achieved = algorithmic bytes per launch / mean
    launch time over all launches of that kernel in the step."""
    fam_time, fam_cases = {}, {}
    for c in cases:
        fam_time[c["family"]] = fam_time.get(c["family"], 0.0) + sum(seconds[(c["matrix"], c["fmt"])])
        fam_cases.setdefault(c["family"], []).append(c)
    total = sum(fam_time.values())
    fam = max(fam_time, key=fam_time.get)
    cs = fam_cases[fam]
    n_launch = sum(len(seconds[(c["matrix"], c["fmt"])]) for c in cs)
    bytes_per_launch = sum(c["bytes"] * len(seconds[(c["matrix"], c["fmt"])]) for c in cs) / n_launch
    achieved = bytes_per_launch / (fam_time[fam] / n_launch) / 1e9
    tr = [traffic.get("%s/%s" % (c["matrix"], c["fmt"])) for c in cs]
    tr_launch = (sum(t * len(seconds[(c["matrix"], c["fmt"])]) for t, c in zip(tr, cs)) / n_launch
                 if tr and all(t is not None for t in tr) else None)
    slow = max(cases, key=lambda c: statistics.mean(seconds[(c["matrix"], c["fmt"])]))
    slow_t = statistics.mean(seconds[(slow["matrix"], slow["fmt"])])
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None if tr_launch is None else round(tr_launch),
            "kernel": FAMILY_LABEL.get(fam, "default CSR kernel on " + fam[4:]), "peak_kind": peak_kind,
            "cases": ["%s/%s" % (c["matrix"], c["fmt"]) for c in cs], "bytes_per_launch": round(bytes_per_launch),
            "share_of_step": round(fam_time[fam] / total, 4),
            "slowest_case": {"case": "%s/%s" % (slow["matrix"], slow["fmt"]),
                             "GBs": round(slow["bytes"] / slow_t / 1e9, 1),
                             "frac": round(slow["bytes"] / slow_t / 1e9 / peak, 4)}}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the SpMV kernels' CUDA sources (the spmv_*.cu files and the
    device headers they include: segmented.cuh, ell.cuh, common.cuh) with
    comments and whitespace removed.  The DRAM counters of a capture are
    valid only for the code they were taken on; the solvers' files and
    comment edits do not change that code."""
    import glob
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2011_08879_gb300", "csrc")
    files = glob.glob(os.path.join(csrc, "spmv_*.cu")) + [os.path.join(csrc, f) for f in
                                                          ("segmented.cuh", "ell.cuh", "common.cuh")]
    for p in sorted(files):
        if os.path.exists(p):
            with open(p, encoding="utf-8") as f:
                src = f.read()
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
            src = re.sub(r"//[^\n]*", " ", src)
            h.update(os.path.basename(p).encode())
            h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profile_traffic(cases, path=None):
    """DRAM bytes per launch of each (matrix, format) case, from the committed
    ncu summary if it was taken on the current kernel sources.  The capture
    runs the quarter-size sweep (same matrix kinds, `--sweep small`) and the
    file records, per kind and format, DRAM bytes over algorithmic bytes
    ('ratio <kind>/<format> <r>'); a streaming kernel's traffic grows in
    proportion to the entries it moves, so the full-size traffic is that
    ratio times the full case's algorithmic bytes."""
    ratios, src = {}, None
    path = path or os.path.join(ROOT, "profiles", "spmv_dram_traffic.txt")
    if os.path.exists(path):
        for line in open(path):
            parts = line.split()
            if len(parts) == 2 and parts[0] == "source":
                src = parts[1]
            if len(parts) == 3 and parts[0] == "ratio":
                ratios[parts[1]] = float(parts[2])
    if src != kernel_source_hash():
        return {}
    out = {}
    for c in cases:
        key = "%s/%s" % (c["matrix"].split("_")[0], c["fmt"])
        if key in ratios:
            out["%s/%s" % (c["matrix"], c["fmt"])] = ratios[key] * c["bytes"]
    return out


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            p = [s.strip() for s in line.split(",")]
            if len(p) == 7:
                self.samples.append((time.perf_counter(), p))

    def window(self, t0, t1, slack=0.06):
        """Keep the samples taken within [t0 - slack, t1 + slack]."""
        inside = [s for s in self.samples if t0 - slack <= s[0] <= t1 + slack]
        self.samples = inside or self.samples[-2:]

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = [s[1] for s in self.samples]
        sm = [float(s[0]) for s in rows if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in rows if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in rows for i in range(4) if s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ CPU baseline

def cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(mats, budget_s=20.0):
    """The oracle's plain CSR SpMV on the sweep matrices, timed twice on the
    host: its row loop on every core of the affinity mask (OpenMP, `value`)
    and the sequential oracle on one thread; each leg as many passes as fit
    in half the budget (at least one per matrix)."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))

    def leg(fn, budget):
        total_b, total_t, passes = 0.0, 0.0, 0
        start = time.perf_counter()
        while True:
            for name, A in mats.items():
                x = syn.vector(A["n_cols"], 99)
                t0 = time.perf_counter()
                fn(A, x)
                total_t += time.perf_counter() - t0
                total_b += spmv_bytes("csr", None, A["n_rows"], A["n_cols"], len(A["val"]))
            passes += 1
            if time.perf_counter() - start > budget:
                break
        return total_b / total_t / 1e9, passes

    v_all, p_all = leg(lambda A, x: oracle.spmv_csr_omp(A, x, cores), budget_s / 2)
    v_one, p_one = leg(oracle.spmv_csr, budget_s / 2)
    return {"value": v_all, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": "%d pass(es) of the oracle's CSR SpMV row loop on %d threads (OpenMP) over the 4 sweep "
                      "matrices" % (p_all, cores),
            "cpu_model": cpu_model(),
            "single_thread": {"value": v_one, "unit": "GB/s", "cores": 1,
                              "sample": "%d pass(es) of the sequential oracle over the 4 sweep matrices" % p_one}}


# -------------------------------------------------------------------- GPU

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate_replicas(bytes_per_rank, seconds, world, device):
    """Whole-job throughput of `world` replicas that each moved
    bytes_per_rank in `seconds`: all ranks' bytes over the slowest rank's
    time (max over ranks through the initialised process group when
    world > 1).  Returns (GB/s, max seconds)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return bytes_per_rank * world / seconds / 1e9, seconds


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_08879_gb300 as gko

    stream = torch.cuda.current_stream()
    st = stream.cuda_stream
    mats, handles = {}, {}
    base = syn.SPMV_SWEEP_SMALL if args.sweep == "small" else SWEEP
    sweep = [m for m in base if not args.only or any(c.split("/")[0] == m for c in args.only.split(","))]
    for name in sweep:
        A = load_workload(name)
        mats[name] = A
        M = gko.Matrix(A, stream=st)
        for f in FORMATS[1:]:
            if args.only and "%s/%s" % (name, f) not in args.only.split(","):
                continue
            try:
                M.convert(f, stream=st)
            except gko.GkoError as e:
                if e.status != gko.binding.ERR_FORMAT_TOO_LARGE:
                    raise
        handles[name] = M
    # (matrix, format) cases with byte counts
    cases = []
    for name, M in handles.items():
        A = mats[name]
        n, m, nnz = A["n_rows"], A["n_cols"], len(A["val"])
        for f in FORMATS:
            if not M.has(f):
                continue
            if args.only and "%s/%s" % (name, f) not in args.only.split(","):
                continue
            info = M.info(f)
            nb = spmv_bytes(f, info, n, m, nnz)
            coo_part = nnz if f in ("csr", "coo") else (info[6] if f == "hybrid" else 0)
            cases.append(dict(matrix=name, fmt=f, bytes=nb, flops=2 * nnz, family=kernel_family(f, name, coo_part),
                              launches=kernel_launches(f, coo_part, csr_launches=csr_default_launches(A))))
    xs = {name: torch.from_numpy(syn.vector(mats[name]["n_cols"], 7)).to(dev) for name in sweep}
    ys = {name: torch.empty(mats[name]["n_rows"], dtype=torch.float64, device=dev) for name in sweep}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def one_step(times):
        for c in cases:
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            handles[c["matrix"]].spmv(xs[c["matrix"]], ys[c["matrix"]], fmt=c["fmt"], stream=st)
            e1.record(stream)
            times.append((c, e0, e1))

    times = []
    # the sampler starts before the warm-up (nvidia-smi needs a moment to
    # produce its first line); only samples inside the timed window are kept
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            one_step([])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            one_step(times)
        torch.cuda.synchronize()
        w1 = time.perf_counter()
        wall = w1 - w0
        time.sleep(0.06)
    clk.window(w0, w1)
    if world > 1:
        torch.distributed.barrier()
    per_case = {}
    for c, e0, e1 in times:
        k = (c["matrix"], c["fmt"])
        per_case.setdefault(k, []).append(e0.elapsed_time(e1) * 1e-3)
    kern_s = sum(sum(v) for v in per_case.values())
    bytes_tot = sum(c["bytes"] for c in cases) * args.steps
    value, kern_s = aggregate_replicas(bytes_tot, kern_s, world, dev)
    peak, peak_kind = measured_peaks()
    detail = {}
    for c in cases:
        ts = per_case[(c["matrix"], c["fmt"])]
        med = statistics.median(ts)
        detail["%s/%s" % (c["matrix"], c["fmt"])] = {
            "GBs": round(c["bytes"] / med / 1e9, 1), "pct_hbm": round(100 * c["bytes"] / med / 1e9 / peak, 1),
            "GFLOPs": round(c["flops"] / med / 1e9, 1), "us": round(med * 1e6, 1)}
    roofline = dominant_roofline(cases, per_case, profile_traffic(cases), peak, peak_kind)

    # end to end through gko_spmv_host with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hx = {n: torch.from_numpy(syn.vector(mats[n]["n_cols"], 7)).pin_memory() for n in sweep}
        hy = {n: torch.empty(mats[n]["n_rows"], dtype=torch.float64).pin_memory() for n in sweep}
        for c in cases:  # warm-up (allocates the staging buffers)
            handles[c["matrix"]].spmv_host(hx[c["matrix"]], hy[c["matrix"]], fmt=c["fmt"], stream=st)
        t_e2e, h2d, d2h = 0.0, 0, 0
        for _ in range(args.steps):
            for c in cases:
                flush.fill_(1.0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                handles[c["matrix"]].spmv_host(hx[c["matrix"]], hy[c["matrix"]], fmt=c["fmt"], stream=st)
                t_e2e += time.perf_counter() - t0
                h2d += 8 * mats[c["matrix"]]["n_cols"]
                d2h += 8 * mats[c["matrix"]]["n_rows"]
        e2e = {"value": round(bytes_tot / t_e2e / 1e9, 1), "unit": "GB/s",
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    extra = {}
    if not args.no_extras and rank == 0:
        extra = run_extras(gko, torch, dev, st, selector=not args.no_selector,
                           selector_matrices=args.selector_matrices)
    launches = sum(c["launches"] for c in cases) * args.steps
    line = {
        "metric": "FP64 SpMV GB/s (algorithmic bytes: values + indices + x + y), all formats x 4 sweep matrices",
        "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(kern_s / args.steps * 1e3, 4), "wall_ms_per_step_incl_flush": round(wall / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64 matrices shaped like the sweep configuration)",
        "config": {"workload": "SpMV sweep: stencil27 128^3 (2.1M rows, 55.7M nnz), banded 4M (bw 64, 16/row), "
                               "power-law 2M (Pareto 1.5, mean 20, max 20k), block-diagonal 1M (8x8)",
                   "formats": "csr (load-balanced), coo, ell (refused where padding > 4 nnz), sellp (S=64), hybrid",
                   "l2": "flushed (512 MB write) before every timed SpMV; inputs also larger than L2 except blockdiag",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "gpu_launches": launches, "e2e": e2e, "detail": detail,
    }
    if rank == 0:
        line["clocks"] = clk.summary()
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(mats, budget_s=args.cpu_budget)
        line["extra"] = extra
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _time_call(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, r


def run_batched_layouts(names):
    """Profiling run: the 4,096-system batched CG solved once in each named
    layout (one kernel launch each, no warm-up), its wall time and status
    printed as one JSON line."""
    import torch
    import paper_2011_08879_gb300 as gko
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    st = torch.cuda.Stream()
    B = load_workload("batched_4096")
    G = gko.Batch(B, stream=st)
    rhs = torch.from_numpy(B["rhs"]).to(dev)
    out = {}
    worst = 0
    for name in names:
        code = gko.binding.batch_layout_code(name)
        x = torch.zeros_like(rhs)
        t, (s, infos) = _time_call(torch, lambda: G.cg(rhs, x, tol=1e-10, maxit=1000, block_size=code, stream=st))
        out[name] = {"s": round(t, 5), "status": s, "max_rel_residual": max(i.rel_residual for i in infos)}
        worst = worst or s
    print(json.dumps({"batched_cg_4096_layouts": out}))
    if worst:
        sys.exit(1)


def run_selector_extra(gko, torch, n_test=200, workers=None):
    """Held-out evaluation of the committed selector on this GPU: the 200
    held-out sweep matrices (seeds 3000..3199) are generated again, every
    candidate is re-timed exactly as the training sweep times it (round
    robin, L2 flushed, median of 5), and the committed network's choice is
    scored against the exhaustive best, the library's default CSR kernel and
    the best fixed candidate of the training set.  Latency: the first
    gko_select_format call on a fresh handle (features + forward)."""
    from paper_2011_08879_gb300 import selector as sel
    w = sel.load()
    params = np.asarray(w["params"], dtype=np.float32)
    mean, scale = np.asarray(w["feat_mean"]), np.asarray(w["feat_scale"])
    seeds = list(range(3000, 3000 + n_test))
    if workers is None:
        workers = max(1, min(14, len(os.sched_getaffinity(0)) - 2))
    t0 = time.perf_counter()
    lat = []

    def on_handle(M):
        if len(lat) < 40:
            torch.cuda.synchronize()
            a = time.perf_counter()
            M.select_format()
            lat.append(time.perf_counter() - a)

    F, T, N, S, worst = sel.sweep(seeds, workers=workers, on_handle=on_handle)
    rep = sel.evaluate(params, mean, scale, F, T)
    fixed_name = w["report"]["test"].get("fixed_best_class")
    fixed = sel.CLASS_NAMES.index(fixed_name) if fixed_name in sel.CLASS_NAMES else None
    exhaustive_s = float(np.nansum(T))  # one timing of every candidate of every matrix
    out = {"matrices": len(seeds), "seeds": "3000..%d" % (3000 + n_test - 1),
           "regret_mean": round(rep["mean"], 4), "regret_median": round(rep["median"], 4),
           "regret_p90": round(rep["p90"], 4), "regret_max": round(rep["max"], 4),
           "default_csr_regret_mean": round(rep["csr_default_mean"], 4),
           "choices": rep["choices"], "structures": {k: S.count(k) for k in sorted(set(S))},
           "max_candidate_disagreement": worst,
           "selector_latency_us_median": round(1e6 * statistics.median(lat), 1) if lat else None,
           "exhaustive_one_timing_per_candidate_ms": round(1e3 * exhaustive_s / len(seeds), 3),
           "wall_s": round(time.perf_counter() - t0, 1),
           "weights_trained_on": "%d matrices" % w["report"].get("n_train", 0)}
    if fixed is not None:
        out["fixed_best_class"] = fixed_name
        out["fixed_best_regret_mean"] = round(float(sel.regret(T, np.full(len(T), fixed)).mean()), 4)
    return out


def run_extras(gko, torch, dev, st, selector=True, selector_matrices=200):
    """CG time to 1e-10 (FP64 and mixed), batched CG, hardware ceilings and
    the selector's held-out regret; outside the timed SpMV region.  Each
    solve runs once untimed first."""
    out = {}
    if selector:
        out["selector"] = run_selector_extra(gko, torch, n_test=selector_matrices)
    L = load_workload("laplace2d_128")
    n = L["n_rows"]
    M = gko.Matrix(L, stream=st)
    xt = torch.from_numpy(syn.vector(n, 1)).to(dev)
    b = torch.empty_like(xt)
    M.spmv(xt, b, stream=st)
    for _ in range(2):
        x = torch.zeros_like(b)
        t, info = _time_call(torch, lambda: M.cg(b, x, tol=1e-10, maxit=10000, stream=st))
    out["cg_laplace2d_128"] = {"s": round(t, 5), "iterations": info.iterations, "rel_residual": info.rel_residual,
                               "status": info.status}
    for _ in range(2):
        x = torch.zeros_like(b)
        t, info = _time_call(torch, lambda: M.cg_single_reduction(b, x, tol=1e-10, maxit=10000, stream=st))
    out["cg_single_reduction_laplace2d_128"] = {"s": round(t, 5), "iterations": info.iterations,
                                                "rel_residual": info.rel_residual, "status": info.status}
    D = load_workload("diffusion7_160")
    n = D["n_rows"]
    M = gko.Matrix(D, stream=st)
    xt = torch.from_numpy(syn.vector(n, 6)).to(dev)
    b = torch.empty_like(xt)
    M.spmv(xt, b, stream=st)
    res = {}
    M.convert("ell", stream=st)
    # FP64 CG: Hestenes-Stiefel and single-reduction forms, CSR and ELL products
    for key, solve, fmt in (("fp64", M.cg, "csr"), ("fp64_single_reduction", M.cg_single_reduction, "csr"),
                            ("fp64_ell", M.cg, "ell"), ("fp64_single_reduction_ell", M.cg_single_reduction, "ell"),
                            ("fp64_jacobi_pcg_ell", M.pcg_jacobi, "ell")):
        for _ in range(2):
            x = torch.zeros_like(b)
            t, info = _time_call(torch, lambda: solve(b, x, tol=1e-10, maxit=20000, fmt=fmt, stream=st))
        err = float(torch.linalg.vector_norm(x - xt) / torch.linalg.vector_norm(xt))
        res[key] = {"s": round(t, 4), "iterations": info.iterations, "rel_residual": info.rel_residual,
                    "status": info.status, "rel_error_vs_x_true": err}
    # block-Jacobi PCG: blocks of up to 8 / 32 consecutive rows (along x on
    # this grid ordering); set-up (supervariables + inversions) timed apart
    for bs in (8, 32):
        for _ in range(2):
            t_setup, P = _time_call(torch, lambda: gko.BlockJacobi(M, bs, stream=st))
            x = torch.zeros_like(b)
            t, info = _time_call(torch, lambda: M.pcg_block_jacobi(P, b, x, tol=1e-10, maxit=20000, fmt="ell",
                                                                   stream=st))
        err = float(torch.linalg.vector_norm(x - xt) / torch.linalg.vector_norm(xt))
        res["fp64_block_jacobi%d_pcg_ell" % bs] = {
            "s": round(t, 4), "setup_s": round(t_setup, 4), "iterations": info.iterations,
            "rel_residual": info.rel_residual, "status": info.status, "rel_error_vs_x_true": err,
            "us_per_iteration": round(t / max(info.iterations, 1) * 1e6, 1)}
        P.close()
    # several right-hand sides: 8 columns sharing one SpMM per step against 8
    # single-vector CG runs (CSR products), 200 steps each (tol 0: no stop)
    kr, steps = 8, 200
    Xt8 = torch.stack([torch.from_numpy(syn.vector(n, 40 + c)).to(dev) for c in range(kr)], dim=1).contiguous()
    B8 = torch.empty_like(Xt8)
    M.spmm(Xt8, B8, stream=st)
    for _ in range(2):
        X8 = torch.zeros_like(B8)
        t_multi, (s8, inf8) = _time_call(torch, lambda: M.cg_multi(B8, X8, tol=0.0, maxit=steps, stream=st))
    cols = [B8[:, c].contiguous() for c in range(kr)]
    for _ in range(2):
        xs = [torch.zeros(n, dtype=torch.float64, device=dev) for _c in range(kr)]
        t_single, _r = _time_call(torch, lambda: [M.cg(cols[c], xs[c], tol=0.0, maxit=steps, fmt="csr", stream=st)
                                                 for c in range(kr)])
    res["cg_multi_rhs8_csr_200_steps"] = {
        "s": round(t_multi, 4), "eight_single_cg_s": round(t_single, 4),
        "speedup": round(t_single / t_multi, 3), "steps": [inf8[c].iterations for c in range(kr)],
        "us_per_step": round(t_multi / steps * 1e6, 1)}
    # mixed: inner tolerances chosen by measurement (FP32 1e-2, BF16 1e-1),
    # without and with the Jacobi-preconditioned inner solve
    for key, prec, itol, pc in (("fp32", "fp32", 1e-2, "none"), ("bf16", "bf16", 1e-1, "none"),
                                ("fp32_jacobi", "fp32", 1e-2, "jacobi"), ("bf16_jacobi", "bf16", 1e-1, "jacobi")):
        for _ in range(2):
            x = torch.zeros_like(b)
            t, info = _time_call(torch, lambda: M.cg_mixed(b, x, inner=prec, tol=1e-10, inner_tol=itol,
                                                           maxit_outer=60, stream=st, precond=pc))
        err = float(torch.linalg.vector_norm(x - xt) / torch.linalg.vector_norm(xt))
        res[key] = {"s": round(t, 4), "inner_tol": itol, "outer": info.outer_iterations,
                    "inner_iterations": info.iterations, "rel_residual": info.rel_residual, "status": info.status,
                    "rel_error_vs_x_true": err}
    # roofline of the Hestenes-Stiefel step on ELL: the product with p.q
    # (slots + p + q), r -= alpha q (r, q, r'), x += alpha p and
    # p = r + beta p (x, p, r, x', p'): 12 slots + 10 vector passes of 8n
    info = M.info("ell")
    step_bytes = 12.0 * info[6] + 80.0 * n
    hs = res["fp64_ell"]
    t_step = hs["s"] / max(hs["iterations"], 1)
    hbm, _kind = measured_peaks()
    hs.update({"us_per_iteration": round(t_step * 1e6, 1), "bytes_per_iteration": int(step_bytes),
               "GBs": round(step_bytes / t_step / 1e9, 1), "frac_hbm": round(step_bytes / t_step / 1e9 / hbm, 3)})
    plain64 = min(res[k]["s"] for k in res if k.startswith("fp64") and "jacobi" not in k)
    res["best_plain_fp64_cg_s"] = plain64
    res["speedup_fp32_vs_plain_fp64_cg"] = round(plain64 / res["fp32"]["s"], 3)
    res["speedup_bf16_vs_plain_fp64_cg"] = round(plain64 / res["bf16"]["s"], 3)
    res["speedup_fp32_jacobi_vs_fp64_jacobi_pcg"] = round(res["fp64_jacobi_pcg_ell"]["s"] / res["fp32_jacobi"]["s"], 3)
    res["speedup_bf16_jacobi_vs_fp64_jacobi_pcg"] = round(res["fp64_jacobi_pcg_ell"]["s"] / res["bf16_jacobi"]["s"], 3)
    out["cg_diffusion7_160"] = res
    # multi-RHS SpMM (k = 8) on the 27-point stencil against 8 SpMVs
    S = load_workload("stencil27_128")
    M = gko.Matrix(S, stream=st)
    k = 8
    Xb = torch.rand((S["n_cols"], k), dtype=torch.float64, device=dev)
    Yb = torch.empty((S["n_rows"], k), dtype=torch.float64, device=dev)
    xs1 = [Xb[:, c].contiguous() for c in range(k)]
    y1 = torch.empty(S["n_rows"], dtype=torch.float64, device=dev)
    for _ in range(3):
        M.spmm(Xb, Yb, stream=st)
    ts, t8 = [], []
    for _ in range(5):
        t, _r = _time_call(torch, lambda: M.spmm(Xb, Yb, stream=st))
        ts.append(t)
        t, _r = _time_call(torch, lambda: [M.spmv(xs1[c], y1, stream=st) for c in range(k)])
        t8.append(t)
    nnz = len(S["val"])
    t_mm, t_mv = statistics.median(ts), statistics.median(t8)
    out["spmm_stencil27_k8"] = {"s": round(t_mm, 6), "eight_spmv_s": round(t_mv, 6),
                                "speedup_vs_spmv": round(t_mv / t_mm, 3),
                                "fp64_tfma_s": round(nnz * k / t_mm / 1e12, 4),
                                "note": "bound by the FP64 pipe (one FMA per entry and column; see ceilings.fp64_tfma_s)"}
    # BiCGSTAB on a nonsymmetric convection-diffusion operator (1024^2 grid)
    C = syn.convdiff2d(1024, 0.8)
    n = C["n_rows"]
    M = gko.Matrix(C, stream=st)
    M.convert("ell", stream=st)
    xt = torch.from_numpy(syn.vector(n, 8)).to(dev)
    b = torch.empty_like(xt)
    M.spmv(xt, b, stream=st)
    res = {}
    for fmt in ("csr", "ell"):
        for _ in range(2):
            x = torch.zeros_like(b)
            t, info = _time_call(torch, lambda: M.bicgstab(b, x, tol=1e-10, maxit=20000, fmt=fmt, stream=st))
        res[fmt] = {"s": round(t, 4), "steps": info.iterations, "rel_residual": info.rel_residual,
                    "status": info.status}
    out["bicgstab_convdiff2d_1024"] = res
    for _ in range(2):
        x = torch.zeros_like(b)
        t, info = _time_call(torch, lambda: M.gmres(b, x, tol=1e-10, restart=30, maxit=20000, fmt="ell", stream=st))
    out["gmres30_convdiff2d_1024"] = {"s": round(t, 4), "steps": info.iterations, "rel_residual": info.rel_residual,
                                      "status": info.status}
    B = load_workload("batched_4096")
    G = gko.Batch(B, stream=st)
    rhs = torch.from_numpy(B["rhs"]).to(dev)
    x = torch.zeros_like(rhs)
    best = G.autotune(rhs, x, stream=st)
    for _ in range(2):
        x = torch.zeros_like(rhs)
        t, (s, infos) = _time_call(torch, lambda: G.cg(rhs, x, tol=1e-10, maxit=1000, stream=st))
    its = [i.iterations for i in infos]
    # other layouts of the autotuner's space, timed on their own for the record
    alt = {}
    P, PQ = gko.binding.BATCH_SHARED_P, gko.binding.BATCH_SHARED_PQ
    for bs_alt in (64, 128, -128, P | 64, P | 128, PQ | 128, P | 256):
        for _ in range(2):
            x2 = torch.zeros_like(rhs)
            t_alt, _r = _time_call(torch, lambda: G.cg(rhs, x2, tol=1e-10, maxit=1000, block_size=bs_alt, stream=st))
        alt[gko.binding.batch_layout(bs_alt)] = round(t_alt, 5)
    # roofline of the batched solve: every iteration re-streams the system's
    # CSR (values + indices + row pointers); vectors live in shared memory
    # or a per-block scratch, depending on the layout (not counted).
    # FP64 work per iteration and row: the product's FMAs plus five vector
    # FMAs (p.q, x, r, r.r, p)
    ro, rp = B["row_off"], B["row_ptr"].astype(np.int64)
    n_s = np.diff(ro)
    nnz_s = rp[ro[1:]] - rp[ro[:-1]]
    its_a = np.array(its, dtype=np.float64)
    mat_bytes = float(np.sum(its_a * (12.0 * nnz_s + 4.0 * (n_s + 1))))
    fmas = float(np.sum(its_a * (nnz_s + 5.0 * n_s)))
    out["batched_cg_4096"] = {"s": round(t, 5), "status": s, "layout": gko.binding.batch_layout(best),
                              "max_rel_residual": max(i.rel_residual for i in infos),
                              "iterations_mean": round(float(np.mean(its)), 2),
                              "matrix_GBs": round(mat_bytes / t / 1e9, 1),
                              "s_by_layout": alt,
                              "fp64_tfma_s": round(fmas / t / 1e12, 4)}
    # hardware ceilings of this GPU (FP64 / FP32 FMA rate, random gathers)
    f64, f32, g16 = gko.binding.gko_measure_ceilings(1 << 21, st)
    g64 = gko.binding.gko_measure_ceilings(1 << 23, st)[2]
    out["ceilings"] = {"fp64_tfma_s": round(f64, 4), "fp32_tfma_s": round(f32, 3),
                       "random_gathers_G_s_x_16MB": round(g16, 1), "random_gathers_G_s_x_64MB": round(g64, 1),
                       "how": "gko_measure_ceilings: 8 FMA chains per thread, 8 blocks of 256 per SM; random 8-byte "
                              "loads from a 16 MB / 64 MB array; best of 5 after a warm-up"}
    out["batched_cg_4096"]["fp64_pipe_frac"] = round(fmas / t / 1e12 / f64, 4)
    return out


# -------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    mats = {name: load_workload(name) for name in SWEEP}
    # one step = the oracle's SpMV of every format on a bounded row sample of
    # each matrix (the first rows holding ~2M entries)
    sample = {}
    for name, A in mats.items():
        rp = A["row_ptr"]
        r1 = int(np.searchsorted(rp, 2_000_000))
        r1 = max(1, min(r1, A["n_rows"]))
        sub = dict(n_rows=r1, n_cols=A["n_cols"], row_ptr=rp[:r1 + 1].copy(), col_idx=A["col_idx"][:rp[r1]],
                   val=A["val"][:rp[r1]])
        conv = {"csr": None, "coo": oracle.to_coo(sub), "sellp": oracle.to_sellp(sub, 64), "hybrid": oracle.to_hybrid(sub)}
        if oracle.max_row_len(sub) * oracle.ell_n_pad(r1) <= max(4 * len(sub["val"]), 1 << 22):
            conv["ell"] = oracle.to_ell(sub)
        sample[name] = (sub, conv)

    def step():
        b = 0.0
        for name, (sub, conv) in sample.items():
            n, m, nnz = sub["n_rows"], sub["n_cols"], len(sub["val"])
            x = syn.vector(m, 7)
            for f, c in conv.items():
                if f == "csr":
                    oracle.spmv_csr(sub, x)
                    info = None
                elif f == "coo":
                    oracle.spmv_coo(n, c, x)
                    info = None
                elif f == "ell":
                    oracle.spmv_ell(n, c, x)
                    info = [1, n, m, nnz, c["K"], c["n_pad"], c["K"] * c["n_pad"], 0]
                elif f == "sellp":
                    oracle.spmv_sellp(n, c, x)
                    info = [1, n, m, nnz, 64, len(c["slice_len"]), len(c["col"]), 1]
                else:
                    oracle.spmv_hybrid(n, c, x)
                    info = [1, n, m, nnz, c["K"], c["n_pad"], len(c["coo_val"]), 0]
                b += spmv_bytes(f, info, n, m, nnz)
        return b

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    tot = 0.0
    for _ in range(args.steps):
        tot += step()
    dt = time.perf_counter() - t0
    v = tot / dt / 1e9
    line = {"impl": "reference", "metric": "FP64 SpMV GB/s (algorithmic bytes: values + indices + x + y), "
            "all formats x 4 sweep matrices", "value": round(v, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "SpMV sweep (same matrices); each step runs every format on the first rows "
                                   "of each matrix holding ~2M stored entries"},
            "cpu_baseline": {"value": round(v, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "first ~2M stored entries of each sweep matrix, every format"},
            "e2e": {"value": round(v, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gko", choices=["gko", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--only", default="", help="comma list of matrix/format cases to time (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-selector", action="store_true", help="skip the selector's held-out re-timing")
    ap.add_argument("--selector-matrices", type=int, default=200,
                    help="held-out matrices re-timed for the selector's regret (seeds 3000 onwards)")
    ap.add_argument("--batched", default="",
                    help="profiling run: only the 4,096-system batched CG, once per layout of this comma list "
                         "(e.g. shared_xrpq/64,shared_p/128)")
    ap.add_argument("--sweep", default="full", choices=["full", "small"],
                    help="small: quarter-size matrices of the same four kinds (profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gko":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.batched:
        run_batched_layouts(args.batched.split(","))
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
