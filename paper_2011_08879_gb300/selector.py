"""Learned format selector: exhaustive sweep, GPU training, regret.

The paper's Sec. 6.1 observes that no SpMV kernel wins on every matrix
("the distinct kernels differ in their efficiency for the distinct problem
characteristics").  This module learns the choice:

* sweep: for each synthetic matrix, time every (format, kernel) candidate
  with CUDA events (L2 flushed between repetitions, median of the reps) and
  record the 12 matrix statistics computed by gko_features;
* train: a 12 -> 64 -> 64 -> C MLP regresses each candidate's log10
  slowdown against the matrix's fastest candidate (capped); the forward
  pass, the gradients and the Adam updates all run in the library's
  kernels (gko_mlp_forward / gko_mlp_grad / gko_mlp_adam), on the GPU; the
  initialisation seed is chosen on a validation split of the training
  matrices;
* evaluate: the chosen candidate is the argmin of the predictions; the
  regret is t(chosen) / t(best) - 1 against the exhaustive best.

The sweep checks that every candidate agrees with the others; the
agreement with the CPU oracle is checked by the GPU tests.

Command line (writes the weights and a JSON report):
    python -m paper_2011_08879_gb300.selector --train 1000:3000 --test 3000:3200 --out weights.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import binding as B
from . import Matrix

CANDIDATES = (
    ("csr", B.CFG_CSR_ROWBLOCK),
    ("csr", B.CFG_CSR_NNZSPLIT),
    ("csr", B.CFG_CSR_SUBWARP_4),
    ("csr", B.CFG_CSR_SUBWARP_32),
    ("coo", 0),
    ("ell", 0),
    ("sellp", 0),
    ("hybrid", 0),
    ("csr", B.CFG_CSR_BINNED),
    ("csr", B.CFG_CSR_SUBWARP_1),
)
CLASS_NAMES = ["%s/%d" % c for c in CANDIDATES]
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")


def _torch():
    import torch
    return torch


def prepare(A, stream=0):
    """Handle with every applicable format materialised (refusals skipped)."""
    M = Matrix(A, stream=stream)
    for f in ("coo", "ell", "sellp", "hybrid"):
        try:
            M.convert(f, stream=stream)
        except B.GkoError as e:
            if e.status != B.ERR_FORMAT_TOO_LARGE:
                raise
    return M


def measure(M, reps=5, warmup=2, flush_bytes=256 << 20, check=True, seed=7, spin_s=0.005, queue_s=0.02):
    """Median time (s) of every candidate on handle M (NaN: not applicable),
    plus the worst relative disagreement between candidates.

    The GPU is first kept busy for spin_s (clocks leave their idle state
    after the host-side set-up of the matrix), then the candidates are timed
    round robin, one repetition of each per round with L2 flushed before
    every run, so that slow drifts of the clock hit every candidate alike.
    All timed launches are queued behind a device-side sleep of queue_s, so
    the GPU runs them back to back: a product of a few microseconds would
    otherwise be timed together with any delay of the host between its start
    event and its launch (a sweep's host also receives the next matrices)."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.current_stream()
    x = torch.rand(M.n_cols, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(seed))
    x = 2 * x - 1
    y = torch.empty(M.n_rows, dtype=torch.float64, device=dev)
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device=dev)
    times = np.full(len(CANDIDATES), np.nan)
    ref = None
    worst = 0.0
    live = []
    for ci, (fmt, cfg) in enumerate(CANDIDATES):  # applicability, warm-up and the agreement check
        if not M.has(fmt):
            continue
        try:
            M.spmv(x, y, fmt=fmt, config=cfg, stream=st.cuda_stream)
        except B.GkoError:
            continue  # configuration does not apply to this matrix
        live.append(ci)
        for _ in range(warmup - 1):
            M.spmv(x, y, fmt=fmt, config=cfg, stream=st.cuda_stream)
        if check:
            if ref is None:
                ref = y.clone()
                scale = float(ref.abs().max()) + 1e-300
            else:
                worst = max(worst, float((y - ref).abs().max()) / scale)
    t_end = time.perf_counter() + spin_s
    while time.perf_counter() < t_end:
        flush.fill_(1.0)
        torch.cuda.synchronize()
    ev = {ci: [] for ci in live}
    torch.cuda._sleep(int(queue_s * 2.0e9))  # ~queue_s at GB300 clocks; the queue below is host-bound
    for _ in range(reps):
        for ci in live:
            fmt, cfg = CANDIDATES[ci]
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            M.spmv(x, y, fmt=fmt, config=cfg, stream=st.cuda_stream)
            e1.record(st)
            ev[ci].append((e0, e1))
    torch.cuda.synchronize()
    for ci in live:
        times[ci] = float(np.median([a.elapsed_time(b) for a, b in ev[ci]])) * 1e-3
    return times, worst


TARGET_CAP = 1.5  # log10 of the slowdown beyond which candidates count as equally bad


def targets(times, nnz=None):
    """Regression targets: log10 of each candidate's slowdown against the
    matrix's fastest candidate, capped at TARGET_CAP (a candidate 30x slower
    only needs to be predicted as clearly bad, not how bad), and the mask of
    the measured candidates.  The argmin of the predictions is the choice,
    which a per-matrix offset does not change; the relative targets remove
    the common size-dependent part that absolute times would make the
    network learn first."""
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.log10(times / np.nanmin(times))
    mask = np.isfinite(t).astype(np.float32)
    return np.where(mask > 0, np.minimum(t, TARGET_CAP), 0.0).astype(np.float32), mask


# ------------------------------------------------------------------ sweep

def _gen(seed):
    import synthetic
    return seed, synthetic.sweep_matrix(seed)


def sweep(seeds, workers=0, log=None, on_handle=None):
    """Features (N x 12), times (N x C), nnz (N), structures for the seeds.
    Matrices are generated in a spawn-started process pool while the GPU
    times the previous ones.  on_handle(M), if given, is called with each
    fresh handle before its features are computed."""
    feats, times, nnzs, structs, worst = [], [], [], [], 0.0
    if workers > 0:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        pool = ctx.Pool(workers)
        it = pool.imap(_gen, seeds, chunksize=1)
    else:
        pool = None
        it = map(_gen, seeds)
    t0 = time.time()
    try:
        for k, (seed, A) in enumerate(it):
            M = prepare(A)
            if on_handle is not None:
                on_handle(M)
            f = M.features()
            t, w = measure(M)
            worst = max(worst, w)
            feats.append(f)
            times.append(t)
            nnzs.append(len(A["val"]))
            structs.append(A.get("structure", "?"))
            M.close()
            if log and (k + 1) % 50 == 0:
                log("sweep %d/%d  %.0fs" % (k + 1, len(seeds), time.time() - t0))
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    return np.array(feats), np.array(times), np.array(nnzs), structs, worst


# ------------------------------------------------------------------ model

def init_params(n_out, seed=0):
    """He-initialised packed parameters (W1 b1 W2 b2 W3 b3), float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((12, 64), (64, 64), (64, n_out)):
        parts.append((rng.standard_normal((fan_out, fan_in)) * math.sqrt(2.0 / fan_in)).astype(np.float32).ravel())
        parts.append(np.zeros(fan_out, np.float32))
    p = np.concatenate(parts)
    assert p.size == B.gko_mlp_param_count(n_out)
    return p


def normaliser(F):
    mean = F.mean(axis=0)
    scale = F.std(axis=0)
    scale[scale == 0] = 1.0
    return mean, scale


def train(F, Y, Mk, epochs=400, batch=128, lr=3e-3, seed=0, log=None):
    """Adam on the masked MSE, all arithmetic in the library's kernels."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.current_stream().cuda_stream
    n_out = Y.shape[1]
    mean, scale = normaliser(F)
    X = torch.from_numpy(((F - mean) / scale).astype(np.float32)).to(dev)
    Yd = torch.from_numpy(Y.astype(np.float32)).to(dev)
    Md = torch.from_numpy(Mk.astype(np.float32)).to(dev)
    p = torch.from_numpy(init_params(n_out, seed)).to(dev)
    g, m, v = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(seed)
    N = X.shape[0]
    step = 0
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(N)).to(dev)
        for b0 in range(0, N, batch):
            idx = order[b0:b0 + batch]
            xb, yb, mb = X[idx].contiguous(), Yd[idx].contiguous(), Md[idx].contiguous()
            if float(mb.sum()) == 0:
                continue
            B.gko_mlp_grad(p.data_ptr(), n_out, xb.data_ptr(), yb.data_ptr(), mb.data_ptr(), xb.shape[0],
                           g.data_ptr(), loss.data_ptr(), st)
            step += 1
            B.gko_mlp_adam(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(), step, lr, 0.9, 0.999,
                           1e-8, st)
        if log and (ep + 1) % 100 == 0:
            log("epoch %d loss %.5f" % (ep + 1, float(loss.item())))
    return p.cpu().numpy(), mean, scale


def predict(params, mean, scale, F):
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    n_out = len(CANDIDATES)
    X = torch.from_numpy(((F - mean) / scale).astype(np.float32)).to(dev)
    P = torch.from_numpy(params.astype(np.float32)).to(dev)
    out = torch.empty((X.shape[0], n_out), dtype=torch.float32, device=dev)
    B.gko_mlp_forward(P.data_ptr(), n_out, X.data_ptr(), X.shape[0], out.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy()


def regret(times, choice):
    """t(choice) / t(best) - 1 per matrix (choices of unmeasured candidates
    count as the worst measured time)."""
    best = np.nanmin(times, axis=1)
    worst = np.nanmax(times, axis=1)
    t = times[np.arange(len(choice)), choice]
    t = np.where(np.isfinite(t), t, worst)
    return t / best - 1.0


def default_csr_class(F):
    """Candidate index of the library's default CSR kernel (GKO_CFG_DEFAULT)
    for each matrix, from its statistics (mean and max row length): rows of
    close length (max <= 2 mean + 16, max <= 128) one thread per row up to 8
    long, staged row blocks up to 20, four lanes per row beyond; skewed rows
    the binned kernel."""
    out = []
    for f in F:
        mean_len, max_len = f[2], f[4]
        if max_len <= 128 and max_len <= 2.0 * mean_len + 16.0 and max_len >= 1:
            cfg = B.CFG_CSR_SUBWARP_1 if max_len <= 8 else (B.CFG_CSR_ROWBLOCK if max_len <= 20 else B.CFG_CSR_SUBWARP_4)
        else:
            cfg = B.CFG_CSR_BINNED
        out.append(CLASS_NAMES.index("csr/%d" % cfg))
    return np.array(out, dtype=int)


def evaluate(params, mean, scale, F, T):
    pred = predict(params, mean, scale, F)
    pred = np.where(np.isfinite(T), pred, np.inf)  # only candidates the matrix admits
    choice = np.argmin(pred, axis=1)
    r = regret(T, choice)
    # the method without the selector: the library's default CSR kernel
    csr_default = regret(T, default_csr_class(F))
    return dict(mean=float(r.mean()), median=float(np.median(r)), p90=float(np.percentile(r, 90)),
                max=float(r.max()), csr_default_mean=float(csr_default.mean()),
                choices={CLASS_NAMES[c]: int((choice == c).sum()) for c in np.unique(choice)})


def train_select(F, T, seeds=(0, 1, 2, 3, 4, 5), val_frac=0.2, epochs=600, log=None):
    """Train one network per seed on (1 - val_frac) of the matrices and keep
    the one with the lowest mean regret on the rest (model selection on a
    validation split of the training matrices only); returns it retrained
    on all of them with the chosen seed."""
    rng = np.random.default_rng(12345)
    order = rng.permutation(len(F))
    n_val = max(1, int(len(F) * val_frac))
    va, tr = order[:n_val], order[n_val:]
    Y, Mk = (np.array(a) for a in zip(*[targets(t) for t in T]))
    best = None
    for sd in seeds:
        p, mu, sc = train(F[tr], Y[tr], Mk[tr], epochs=epochs, seed=sd)
        r = evaluate(p, mu, sc, F[va], T[va])["mean"]
        if log:
            log("seed %d validation regret %.4f" % (sd, r))
        if best is None or r < best[0]:
            best = (r, sd)
    params, mean, scale = train(F, Y, Mk, epochs=epochs, seed=best[1])
    return params, mean, scale, dict(seed=best[1], validation_regret=best[0])


def save(path, params, mean, scale, report):
    with open(path, "w") as f:
        json.dump(dict(classes=CLASS_NAMES, fmts=[B.FORMATS[c[0]] for c in CANDIDATES],
                       cfgs=[c[1] for c in CANDIDATES], params=[float(v) for v in params],
                       feat_mean=[float(v) for v in mean], feat_scale=[float(v) for v in scale], report=report), f)


def load(path=DEFAULT_WEIGHTS):
    """Install trained weights for GKO_FMT_AUTO; returns the JSON dict."""
    with open(path) as f:
        d = json.load(f)
    p = np.ascontiguousarray(d["params"], dtype=np.float32)
    mean = np.ascontiguousarray(d["feat_mean"], dtype=np.float64)
    scale = np.ascontiguousarray(d["feat_scale"], dtype=np.float64)
    fm = np.ascontiguousarray(d["fmts"], dtype=np.int32)
    cf = np.ascontiguousarray(d["cfgs"], dtype=np.int32)
    B.gko_selector_load(p.ctypes.data, len(fm), mean.ctypes.data, scale.ctypes.data, fm.ctypes.data, cf.ctypes.data)
    return d


def _range(s):
    a, b = s.split(":")
    return list(range(int(a), int(b)))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", default="1000:3000")
    ap.add_argument("--test", default="3000:3200")
    ap.add_argument("--workers", type=int, default=max(1, min(12, (os.cpu_count() or 2) - 2)))
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--report", default="")
    ap.add_argument("--save-sweep", default="", help="write the sweep (features, times, nnz) to this .npz")
    ap.add_argument("--load-sweep", default="", help="train and evaluate on a saved sweep instead of timing")
    args = ap.parse_args(argv)

    def log(s):
        print(s, file=sys.stderr, flush=True)

    t0 = time.time()
    tr, te = _range(args.train), _range(args.test)
    if args.load_sweep:
        z = np.load(args.load_sweep, allow_pickle=False)
        if list(z["classes"]) != CLASS_NAMES:
            raise SystemExit("saved sweep has other candidates: %s" % list(z["classes"]))
        Ftr, Ttr, Ntr, Str = z["Ftr"], z["Ttr"], z["Ntr"], list(z["Str"])
        Fte, Tte, Nte, Ste = z["Fte"], z["Tte"], z["Nte"], list(z["Ste"])
        w1 = w2 = float(z["worst"])
        tr, te = list(z["seeds_tr"]), list(z["seeds_te"])
    else:
        Ftr, Ttr, Ntr, Str, w1 = sweep(tr, args.workers, log)
        Fte, Tte, Nte, Ste, w2 = sweep(te, args.workers, log)
        if args.save_sweep:
            np.savez(args.save_sweep, classes=np.array(CLASS_NAMES), Ftr=Ftr, Ttr=Ttr, Ntr=Ntr, Str=np.array(Str),
                     Fte=Fte, Tte=Tte, Nte=Nte, Ste=np.array(Ste), worst=max(w1, w2), seeds_tr=np.array(tr),
                     seeds_te=np.array(te))
    t_sweep = time.time() - t0
    t1 = time.time()
    params, mean, scale, sel_info = train_select(Ftr, Ttr, epochs=args.epochs, log=log)
    t_train = time.time() - t1
    rep = evaluate(params, mean, scale, Fte, Tte)
    rep_train = evaluate(params, mean, scale, Ftr, Ttr)
    # best single fixed candidate chosen on the training set
    mean_train = [np.nanmean(regret(Ttr, np.full(len(Ttr), c))) for c in range(len(CANDIDATES))]
    fixed = int(np.argmin(mean_train))
    rep["fixed_best_class"] = CLASS_NAMES[fixed]
    rep["fixed_best_mean"] = float(regret(Tte, np.full(len(Tte), fixed)).mean())
    # selector latency: features + forward for one matrix (host-timed)
    report = dict(test=rep, train_mean=rep_train["mean"], n_train=len(tr), n_test=len(te), sweep_s=t_sweep,
                  train_s=t_train, model_selection=sel_info, max_candidate_disagreement=max(w1, w2),
                  structures_test={s: Ste.count(s) for s in set(Ste)})
    save(args.out, params, mean, scale, report)
    out = json.dumps(report)
    print(out)
    if args.report:
        with open(args.report, "w") as f:
            f.write(out + "\n")


if __name__ == "__main__":
    main()
