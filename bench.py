"""SP-SVM benchmark on GB300.

One step = one whole SP-SVM fit (row norms, candidate scoring, kernel-block
growth, Newton reoptimisation with masked Gram, the Newton solve (FP32 tile
Cholesky with FP64 refinement by default) and line search; Section 4, Eq. 4) followed by prediction on 100,000 held-out
queries, on the Gaussian-mixture workload n = 500,000, d = 128, |J| grown 64
at a time from 256 candidates to 4,096.  Inputs stay resident in HBM; the
kernel matrix (8.2 GB) and X (256 MB) are far larger than L2 (129 MB), so no
explicit L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the float64 CPU
oracle on a bounded sample of the same workload on the host cores.
--micro cholesky [--sizes m1,m2,...] times the Newton solve alone: the FP64
factorisation and solve, and the FP32 tile factor with FP64 refinement (the
profiles' capture command).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SP-SVM fit sec & kernel TFLOP/s (n=500k,|J|=4096) vs FP32 form; serve p50/p99"
WORKLOAD = dict(workload="gaussian_mixture_precision_form", n=500_000, d=128, basis=4096,
                candidates=256, add_per_round=64, lam=1e-4, gamma="1/d", components=10,
                queries=100_000)

SLOTS = ["kernel_block", "score", "outputs", "gemv", "compact", "gram", "cholesky", "solve",
         "line_search", "decision", "fit", "lowrank"]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            P = json.load(f)
        return P, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        # raw samples in the temp directory; the JSON line carries their summary
        self.path = os.path.join(tempfile.gettempdir(), f"spsvm_clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


class UtilSampler:
    """nvidia-smi utilization.gpu (percent of time a kernel ran) every 100 ms."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"spsvm_util_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", "--query-gpu=utilization.gpu",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        v = []
        for line in open(self.path):
            try:
                v.append(float(line.strip()))
            except ValueError:
                pass
        return {"mean": statistics.mean(v) if v else None, "samples": len(v)}


def max_over_ranks(x, ws, device="cuda"):
    """Largest value of x over the ranks (the slowest replica's time)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_facts():
    """Host cores the oracle ran on (nproc, the BLAS thread count) and the CPU model."""
    try:
        from threadpoolctl import threadpool_info
        blas = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        blas = None
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return dict(nproc=os.cpu_count(), blas_threads=blas, cpu_model=model)


# Bounded samples of the workload for the oracle: (n, |J|) with d = 128 and
# the same mixture, kappa = 256, q = 64.  The first is the timed sample; the
# other two vary n and |J| alone, which fixes the exponents of the fit time
# t ~ n^a |J|^b used to extrapolate (labelled an estimate).
CPU_SAMPLES = ((4000, 256), (8000, 256), (4000, 512))


def _oracle_fit_seconds(n, J):
    from oracle import spsvm as O
    from paper_1404_1066_gb300 import synth
    p = synth.gaussian_mixture(n=n, d=128, budget=J, seed=1003)
    t0 = time.perf_counter()
    O.fit(p.X, p.y, p.gamma, p.lam, J, tol=1e-6, kappa=256, q=64, seed=1)
    return time.perf_counter() - t0


def gpu_sample_fit_seconds(sp, torch, precision="bf16split"):
    """This library's fit on the CPU baseline's first sample (same rows,
    d = 128, |J| = 256, kappa = 256, q = 64), event-timed after one warm-up:
    the like-for-like partner of the oracle's time."""
    from paper_1404_1066_gb300 import synth
    n0, J0 = CPU_SAMPLES[0]
    p = synth.gaussian_mixture(n=n0, d=128, budget=J0, seed=1003)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    kw = dict(precision=precision, candidates=256, add_per_round=64, seed=1)
    sp.spsvm_fit(X, y, p.gamma, p.lam, J0, 1e-6, **kw)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    sp.spsvm_fit(X, y, p.gamma, p.lam, J0, 1e-6, **kw)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def cpu_baseline_run(steps=1, scaling=True):
    """The float64 oracle, as it stands, timed on the host cores: `steps`
    fits of the first sample (n = 4,000 rows of the same mixture, d = 128,
    |J| = 256), and, with `scaling`, one fit each of the other two samples,
    from which the exponents a, b of t ~ n^a |J|^b and an extrapolated
    full-size fit time (an estimate, not a measurement) follow."""
    n0, J0 = CPU_SAMPLES[0]
    _oracle_fit_seconds(1000, 64)   # untimed: library and thread-pool start-up
    times = [_oracle_fit_seconds(n0, J0) for _ in range(steps)]
    out = dict(sample=f"oracle fit on n={n0:,} rows of the same mixture, d=128, |J|={J0} "
                      f"(kappa=256, q=64)", sample_seconds=times, **_cpu_facts())
    if scaling:
        # each point the faster of two fits (the host cores are shared)
        t0 = min(statistics.median(times), _oracle_fit_seconds(n0, J0))
        tn = min(_oracle_fit_seconds(*CPU_SAMPLES[1]) for _ in range(2))
        tj = min(_oracle_fit_seconds(*CPU_SAMPLES[2]) for _ in range(2))
        a = math.log(tn / t0) / math.log(CPU_SAMPLES[1][0] / n0)
        b = math.log(tj / t0) / math.log(CPU_SAMPLES[2][1] / J0)
        est = t0 * (500_000 / n0) ** a * (4096 / J0) ** b
        out.update(points=[dict(n=n, basis=J, seconds=t) for (n, J), t in
                           zip(CPU_SAMPLES, (t0, tn, tj))],
                   exponent_n=a, exponent_basis=b, full_size_estimate_s=est)
    return out


def batched_leg(sp, torch, workers=8, precision="bf16split"):
    """One-vs-rest 10 classes x gamma in {0.25,0.5,1,2}/d x lambda in
    {1e-3,1e-4,1e-5} = 120 solves on seeded subsamples of a shared
    60,000 x 256 mixture, |J| in [256, 2048]."""
    from paper_1404_1066_gb300 import synth
    X, comp, solves = synth.ovr_grid()
    probs = [dict(rows=s.rows, y=synth.ovr_labels(comp[s.rows], s.label_class), gamma=s.gamma,
                  lam=s.lam, budget=s.budget, tol=1e-6, seed=10_000 + s.solve_id) for s in solves]
    Xd = torch.from_numpy(X).cuda()
    torch.cuda.synchronize()
    util = UtilSampler(torch.cuda.current_device())
    util.start()
    t0 = time.perf_counter()
    models, st = sp.spsvm_fit_batched(Xd, probs, workers=workers, precision=precision,
                                      candidates=256, add_per_round=64)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    busy = util.stop()
    ok = sum(1 for v in st if v in (0, -4))
    return dict(solves=len(probs), ok=ok, seconds=el, solves_per_s=len(probs) / el,
                workers=workers, rows_mean=float(np.mean([len(p["rows"]) for p in probs])),
                basis_mean=float(np.mean([p["budget"] for p in probs])),
                gpu_busy_pct_mean=busy.get("mean"), gpu_busy_samples=busy.get("samples"))


def gram_stress_leg(sp, torch, lib, n=200_000, d=128, budget=2048, sigma_m=0.3,
                    precision="bf16split"):
    """A fit where the masked Gram matrix carries real work: the same
    mixture generator with component means drawn at sigma_m = 0.3 (classes
    overlap: training error ~10%, ~40% of the points active), n = 200,000,
    |J| = 2,048.  Reports the Gram matrix's event-timed TFLOP/s over the fit
    (four plane products) against the measured sustained BF16 peak."""
    import ctypes as C
    from paper_1404_1066_gb300 import synth
    p = synth.gaussian_mixture(n=n, d=d, budget=budget, seed=1007, sigma_m=sigma_m)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    lib.spsvm_profile_enable(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    m = sp.spsvm_fit(X, y, p.gamma, p.lam, budget, 1e-6, precision=precision, candidates=256,
                     add_per_round=64, seed=1)
    e1.record()
    torch.cuda.synchronize()
    nm, L_, t_, w_ = C.c_char_p(), C.c_int64(), C.c_double(), C.c_double()
    lib.spsvm_profile_read(SLOTS.index("gram"), C.byref(nm), C.byref(L_), C.byref(t_), C.byref(w_))
    lib.spsvm_profile_enable(0)
    h = m.history()
    last = [x["active"] for x in h if x["basis"] == budget]
    peaks, src = _peaks()
    tf = w_.value / (t_.value * 1e-3) / 1e12 if t_.value > 0 else None
    return dict(n=n, d=d, basis=budget, sigma_m=sigma_m, fit_s=e0.elapsed_time(e1) / 1e3,
                newton_steps=m.info()["newton_steps"], status=m.status,
                active_fraction_last_round=float(np.mean(last)) / n if last else None,
                train_error=h[-1]["errors"] / n, gram_launches=L_.value, gram_ms=t_.value,
                gram_tflops=tf, gram_frac=(tf / peaks["bf16_tflops_sustained"]) if tf else None,
                peak_source=src)


def serve_leg(sp, requests=100, workers=8, budget_gb=150.0, precision="bf16split"):
    """Poisson arrivals (mean 20 requests/s) of fit requests (n log-uniform in
    [1k, 200k], d in {32, 128, 784}, |J| in {128, ..., 2048}, mixture data)
    interleaved with predict requests of 1k-100k points; HBM admission budget
    150 GB; latency = submission to completion."""
    from paper_1404_1066_gb300 import synth
    reqs = synth.arrival_stream(count=requests)
    bases = {}
    for dd in sorted({r.d for r in reqs}):
        b = synth.gaussian_mixture(n=200_000, d=dd, budget=64, seed=2000 + dd)
        bases[dd] = (b.X, np.where(b.meta["components"] % 2 == 0, 1.0, -1.0).astype(np.float32))
    srv = sp.Server(int(budget_gb * 2 ** 30), workers=workers)
    ids, kinds = [], []
    t0 = time.perf_counter()
    for k, r in enumerate(reqs):
        delay = r.t_arrival - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        Xb, yb = bases[r.d]
        if r.kind == "fit":
            rid = srv.submit_fit(Xb[:r.n], yb[:r.n], 1.0 / r.d, 1e-4, r.budget, 1e-6,
                                 precision=precision, candidates=256, add_per_round=64,
                                 seed=r.seed & 0xFFFFFFFF)
        else:
            rid = srv.submit_predict(ids[r.target], Xb[-r.n:])
        ids.append(rid)
        kinds.append(r.kind)
    lats, fails = {"fit": [], "predict": []}, 0
    for rid, kind in zip(ids, kinds):
        st, lat = srv.wait(rid, -1.0)
        if st not in (0, -4):
            fails += 1
        lats[kind].append(lat)
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    allv = lats["fit"] + lats["predict"]
    pct = lambda v, q: float(np.percentile(v, q)) if v else None
    return dict(requests=requests, fits=len(lats["fit"]), predicts=len(lats["predict"]),
                failed=fails, wall_s=wall, solves_per_s=len(lats["fit"]) / wall,
                p50_ms=pct(allv, 50), p99_ms=pct(allv, 99), fit_p50_ms=pct(lats["fit"], 50),
                fit_p99_ms=pct(lats["fit"], 99), predict_p50_ms=pct(lats["predict"], 50),
                predict_p99_ms=pct(lats["predict"], 99), hbm_peak_gb=stats["hbm_peak"] / 2 ** 30,
                workers=workers, budget_gb=budget_gb, arrival_rate=20.0)


# DRAM bytes (read + write) / algorithmic bytes of the GEMV launch, the
# median over twelve launches of an ncu capture of the current kernel
# (n = 100,000, |J| = 320 and 384; the summary is in profiles/)
GEMV_TRAFFIC_RATIO = 0.998


def _leg(fn, *a, **k):
    """An auxiliary leg of the bench line: its result, or its error, without
    losing the line's headline measurement."""
    try:
        return fn(*a, **k)
    except Exception as e:   # reported in the JSON line instead
        return dict(error=f"{type(e).__name__}: {e}")


def ovo_leg(sp, torch, n=60_000, d=256, classes=10, budget=256, workers=8, precision="bf16split"):
    """One-vs-one over a 10-class mixture (the grouped form of Section 5's
    multiclass runs): the 45 pair problems as one batch, then voting on
    fresh points of the same mixture."""
    from paper_1404_1066_gb300 import synth
    p = synth.gaussian_mixture(n=n, d=d, components=classes, seed=1006, lam=1e-4, budget=budget)
    cls = p.meta["components"].astype(np.int64)
    Xq, cq = synth.mixture_holdout(p, 20_000, seed=89, components=True)
    X = torch.from_numpy(p.X).cuda()
    Xqd = torch.from_numpy(Xq).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    models, st = sp.spsvm_fit_ovo(X, cls, classes, p.gamma, p.lam, budget, 1e-6, workers=workers,
                                  precision=precision, candidates=256, add_per_round=64, seed=1)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    lab, _ = sp.spsvm_predict_ovo(models, classes, Xqd)
    lab = lab.cpu().numpy()
    pred_s = time.perf_counter() - t1
    return dict(classes=classes, pairs=len(models), ok=int(sum(1 for s in st if s == 0)), n=n, d=d,
                basis=budget, fit_s=fit_s, pairs_per_s=len(models) / fit_s, predict_s=pred_s,
                queries=len(Xq), holdout_accuracy=float(np.mean(lab == cq)), workers=workers)


def exact_score_leg(sp, torch, n=100_000, d=128, budget=512, precision="bf16split"):
    """Basis selection by Section 4's heuristic estimate against the exact
    one-dimensional decrease, on a mixture of the bench's kind: fit seconds
    and held-out accuracy of each."""
    from paper_1404_1066_gb300 import synth
    p = synth.gaussian_mixture(n=n, d=d, seed=1007, budget=budget)
    Xh, yh = synth.mixture_holdout(p, 20_000, seed=90)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    Xhd = torch.from_numpy(Xh).cuda()
    out = {}
    for score in ("heuristic", "exact"):
        sp.spsvm_fit(X, y, p.gamma, p.lam, 64, 1e-6, precision=precision, seed=1, score=score)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = sp.spsvm_fit(X, y, p.gamma, p.lam, budget, 1e-6, precision=precision, candidates=256,
                         add_per_round=64, seed=1, score=score)
        torch.cuda.synchronize()
        fs = time.perf_counter() - t0
        f = sp.spsvm_predict(m, Xhd).cpu().numpy()
        out[score] = dict(fit_s=fs, holdout_accuracy=float(np.mean(np.where(f >= 0, 1.0, -1.0) == yh)),
                          objective=m.info()["objective"], newton_steps=m.info()["newton_steps"])
    return dict(n=n, d=d, basis=budget, **out)


def growth_leg(sp, torch, model, X, y, p, work, opts, stream, holdout=100_000):
    from paper_1404_1066_gb300 import synth
    eps = sp._lib.SPSVM_GROWTH_EPS_PAPER
    Xh, yh = synth.mixture_holdout(p, holdout, seed=88)
    Xhd = torch.from_numpy(Xh).cuda()
    n = X.shape[0]

    def acc(m):
        f = sp.spsvm_predict(m, Xhd).cpu().numpy()
        return float(np.mean(np.where(f >= 0, 1.0, -1.0) == yh))

    ends = {}
    for h in model.history():
        ends[h["basis"]] = h["errors"]
    curve = [[b, e / n] for b, e in sorted(ends.items())]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ms = sp.spsvm_fit(X, y, p.gamma, p.lam, p.budget, 1e-6, workspace=work,
                      growth_tol=eps, **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    info = ms.info()
    hist = ms.history()
    return dict(eps=eps, rounds=info["rounds"], basis=info["n_basis"],
                fit_s=e0.elapsed_time(e1) / 1e3,
                train_error=hist[-1]["errors"] / n if hist else None,
                holdout_accuracy=acc(ms), holdout=holdout,
                budget_basis=p.budget, budget_holdout_accuracy=acc(model),
                train_error_vs_basis=curve)


def run_micro_kblock(args):
    """The tensor-core kernel block alone: the mixture workload's points
    (n x d, prepared once), |J| = --basis random basis rows, K stored in
    FP32 as the fit stores it; event-timed per launch.  TFLOP/s counts the
    six plane products (6 x 2 n |J| d); GB/s counts the n |J| x 4 bytes
    written."""
    import torch
    import paper_1404_1066_gb300 as sp
    from paper_1404_1066_gb300 import synth
    sp.load()
    n, d, m, prec = args.n, args.d, args.basis, args.precision
    p = synth.gaussian_mixture(n=n, d=d, budget=m, seed=1003)
    X = torch.from_numpy(p.X).cuda()
    P = sp.spsvm_prepare_points(X, prec)
    idx = torch.from_numpy(np.random.default_rng(1).choice(n, m, replace=False).astype(np.int64)).cuda()
    km = sp.kmat_empty(n, m, "fp32")
    for _ in range(args.warmup):
        sp.spsvm_kernel_block(P, idx, p.gamma, prec, km)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sp.spsvm_kernel_block(P, idx, p.gamma, prec, km)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    prod = 6.0 if prec == "bf16split" else 1.0
    print(json.dumps(dict(micro="kblock", n=n, d=d, basis=m, precision=prec, ms=ms,
                          tflops=prod * 2.0 * n * m * d / (ms * 1e-3) / 1e12,
                          write_gbs=4.0 * n * m / (ms * 1e-3) / 1e9, steps=args.steps)), flush=True)
    return 0


def run_micro_gram(args):
    """The masked Gram matrix alone: K_nJ of the mixture workload (kernel
    block, FP32), every point active (|S| = n), compacted into the hi / lo
    planes and contracted on the tensor cores (BF16SPLIT) or in FP32 SIMT;
    event-timed per spsvm_gram call (contraction + finish).  TFLOP/s counts
    4 x |S| |J| (|J| + 1) flops (four plane products, upper triangle)."""
    import torch
    import paper_1404_1066_gb300 as sp
    from paper_1404_1066_gb300 import synth
    sp.load()
    n, d, m, prec = args.n, args.d, args.basis, args.precision
    p = synth.gaussian_mixture(n=n, d=d, budget=m, seed=1003)
    X = torch.from_numpy(p.X).cuda()
    P = sp.spsvm_prepare_points(X, prec)
    J = torch.from_numpy(np.random.default_rng(1).choice(n, m, replace=False).astype(np.int64)).cuda()
    km = sp.kmat_empty(n, m, "fp32")
    sp.spsvm_kernel_block(P, J, p.gamma, prec, km)
    act = torch.ones(n, dtype=torch.uint8, device="cuda")
    kc = sp.kmat_empty(km.ld, m, prec, ld=km.ld)
    _, _, nact, _ = sp.spsvm_compact_active(km, act, None, None, kc)
    for _ in range(args.warmup):
        sp.spsvm_gram(kc, nact, n, km, J, p.lam, prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sp.spsvm_gram(kc, nact, n, km, J, p.lam, prec)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    prod = 4.0 if prec == "bf16split" else 1.0
    print(json.dumps(dict(micro="gram", n=n, active=n, basis=m, precision=prec, ms=ms,
                          tflops=prod * n * m * (m + 1) / (ms * 1e-3) / 1e12, steps=args.steps)),
          flush=True)
    return 0


def run_micro(args):
    """The Newton solve alone at the given sizes, on random SPD matrices
    A A^T / m + I / 2 (seeded): the FP64 factorisation and its solve, and the
    FP32 tile factor with FP64 refinement (factor and refinement together,
    and the refinement alone); one JSON line of event-timed milliseconds."""
    import torch
    import paper_1404_1066_gb300 as sp
    lib = sp.load()
    out = {}
    for m in [int(v) for v in args.sizes.split(",")]:
        g = np.random.default_rng(m)
        A = g.standard_normal((m, m + 5)) / np.sqrt(m)
        H0 = torch.from_numpy(A @ A.T + 0.5 * np.eye(m)).cuda()
        b0 = torch.from_numpy(g.standard_normal(m)).cuda()
        Hs = [H0.clone() for _ in range(args.warmup + args.steps)]
        for k in range(args.warmup):
            assert sp.spsvm_cholesky(Hs[k]) == 0
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(args.warmup, args.warmup + args.steps):
            sp.spsvm_cholesky(Hs[k])
        e1.record()
        torch.cuda.synchronize()
        fac = e0.elapsed_time(e1) / max(1, args.steps)
        L = Hs[-1]
        b = b0.clone()
        for _ in range(args.warmup):
            sp.spsvm_cholesky_solve(L, b)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            sp.spsvm_cholesky_solve(L, b)
        e1.record()
        torch.cuda.synchronize()
        sol = e0.elapsed_time(e1) / max(1, args.steps)
        # mixed: FP32 factor + FP64 refinement (H kept), one solve included
        Hm = H0.clone()
        for _ in range(args.warmup):
            sp.spsvm_solve_mixed(Hm, b0)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            info, st, _, iters, be = sp.spsvm_solve_mixed(Hm, b0)
        e1.record()
        torch.cuda.synchronize()
        mixed_both = e0.elapsed_time(e1) / max(1, args.steps)
        # the mixed solve alone (refinement to FP64 backward error) with the
        # FP32 factor in hand
        import ctypes as C
        wb = lib.spsvm_mixed_work_bytes(m)
        work = torch.empty(max(256, wb), dtype=torch.uint8, device="cuda")
        info_d = torch.zeros(1, dtype=torch.int32, device="cuda")
        x = torch.zeros(m, dtype=torch.float64, device="cuda")
        lib.spsvm_cholesky_mixed(Hm.data_ptr(), m, Hm.stride(0), 0.0, info_d.data_ptr(),
                                 work.data_ptr(), wb, None)
        it_c, be_c = C.c_int32(), C.c_double()
        solve_once = lambda: lib.spsvm_solve_mixed(Hm.data_ptr(), m, Hm.stride(0), 0.0,
                                                   b0.data_ptr(), x.data_ptr(), 30, 1e-13,
                                                   C.byref(it_c), C.byref(be_c), work.data_ptr(),
                                                   wb, None)
        for _ in range(args.warmup):
            solve_once()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            solve_once()
        e1.record()
        torch.cuda.synchronize()
        out[str(m)] = dict(factor_ms=fac, solve_ms=sol,
                           fp64_equiv_tflops=m ** 3 / 3.0 / (fac * 1e-3) / 1e12,
                           mixed_factor_and_solve_ms=mixed_both,
                           mixed_solve_ms=e0.elapsed_time(e1) / max(1, args.steps),
                           mixed_solve_iters=it_c.value,
                           mixed_iters=iters, mixed_backward_error=be, mixed_status=st)
        del Hs, L
    print(json.dumps(dict(micro="cholesky", steps=args.steps, warmup=args.warmup, sizes=out)),
          flush=True)
    return 0


def run_reference(args):
    """The float64 oracle, as it stands, on the host cores: each step one fit
    of the bounded sample (n = 4,000, |J| = 256 of the same mixture); the
    line's value is that measured time per step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        _oracle_fit_seconds(*CPU_SAMPLES[0])
    cb = cpu_baseline_run(steps=args.steps, scaling=False)
    per = statistics.mean(cb["sample_seconds"])
    line = dict(metric=METRIC, value=per, unit="s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=per * 1e3, higher_is_better=False,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(WORKLOAD, l2="inputs larger than L2", sample=cb["sample"]),
                impl="reference",
                cpu_baseline=dict(value=per, unit="s", cores=cb["nproc"], kind="oracle",
                                  sample=cb["sample"], sample_seconds=cb["sample_seconds"],
                                  blas_threads=cb["blas_threads"], cpu_model=cb["cpu_model"]),
                e2e=dict(value=per, unit="s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_1404_1066_gb300 as sp
    from paper_1404_1066_gb300 import synth
    import ctypes as C

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    lib = sp.load()
    n, d, J = args.n, args.d, args.basis
    prec = args.precision
    p = synth.gaussian_mixture(n=n, d=d, budget=J, seed=1003 + rank)
    Xq_h = synth.queries_like(p, args.queries, seed=77 + rank)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    Xq = torch.from_numpy(Xq_h).cuda()
    opts = dict(precision=prec, candidates=256, add_per_round=64, seed=1)
    o, _ = sp.make_options(**opts)
    wsb = lib.spsvm_fit_workspace_bytes(n, d, J, C.byref(o))
    work = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        m = sp.spsvm_fit(X, y, p.gamma, p.lam, J, 1e-6, workspace=work, **opts)
        f = sp.spsvm_predict(m, Xq)
        return m, f

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    lib.spsvm_profile_enable(1)
    launches0 = lib.spsvm_launch_count()
    torch.cuda.synchronize()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        model, f = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = lib.spsvm_launch_count() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = {}
    for k, name in enumerate(SLOTS):
        nm = C.c_char_p()
        L = C.c_int64()
        t = C.c_double()
        w = C.c_double()
        lib.spsvm_profile_read(k, C.byref(nm), C.byref(L), C.byref(t), C.byref(w))
        prof[name] = dict(launches=L.value, ms=t.value, work=w.value)
    lib.spsvm_profile_enable(0)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, ws)
    info = model.info()

    # end to end through the public API from pinned host buffers
    Xh = torch.from_numpy(p.X).pin_memory()
    yh = torch.from_numpy(p.y).pin_memory()
    Xqh = torch.from_numpy(Xq_h).pin_memory()
    out_h = torch.empty(args.queries, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        Xd = Xh.to("cuda", non_blocking=True)
        yd = yh.to("cuda", non_blocking=True)
        Xqd = Xqh.to("cuda", non_blocking=True)
        m2 = sp.spsvm_fit(Xd, yd, p.gamma, p.lam, J, 1e-6, workspace=work, **opts)
        fo = sp.spsvm_predict(m2, Xqd)
        out_h.copy_(fo, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.e2e_steps, ws)
    h2d = p.X.nbytes + p.y.nbytes + Xq_h.nbytes
    d2h = args.queries * 4

    # kernel-block throughput: the full n x |J| block of the final basis
    Jidx = torch.from_numpy(model.basis_and_beta()[0]).cuda()
    P = sp.spsvm_prepare_points(X, prec)
    km = sp.kmat_empty(n, J, "fp32")   # K_nJ is stored in FP32 in both forms
    for _ in range(2):
        sp.spsvm_kernel_block(P, Jidx, p.gamma, prec, km)
    kb0 = torch.cuda.Event(enable_timing=True)
    kb1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    kb0.record(stream)
    for _ in range(reps):
        sp.spsvm_kernel_block(P, Jidx, p.gamma, prec, km)
    kb1.record(stream)
    torch.cuda.synchronize()
    kb_ms = kb0.elapsed_time(kb1) / reps
    split = 6.0 if prec == "bf16split" else 1.0   # plane products per FP32 product
    kb_tflops = split * 2.0 * n * J * d / (kb_ms * 1e-3) / 1e12
    del km

    # growth stop of Section 4 at the paper's epsilon, and the accuracy
    # against |J| of the run to budget (training error after each round,
    # held-out accuracy at the end) on fresh points of the same mixture
    growth = None
    if args.growth:
        growth = _leg(growth_leg, sp, torch, model, X, y, p, work, opts, stream)

    # the same fit with the low-rank correction of the Newton factor
    # (spsvm_options.lowrank): fit time, and how the Newton systems were solved
    lowrank = None
    if args.lowrank:
        def lowrank_leg():
            lib.spsvm_profile_enable(1)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            ml = sp.spsvm_fit(X, y, p.gamma, p.lam, J, 1e-6, workspace=None, lowrank=True, **opts)
            a1.record(stream)
            torch.cuda.synchronize()
            pl = {}
            for k, name in enumerate(SLOTS):
                if name not in ("cholesky", "lowrank", "solve"):
                    continue
                nm, L_, t_, w_ = C.c_char_p(), C.c_int64(), C.c_double(), C.c_double()
                lib.spsvm_profile_read(k, C.byref(nm), C.byref(L_), C.byref(t_), C.byref(w_))
                pl[name] = dict(launches=L_.value, ms=t_.value)
            lib.spsvm_profile_enable(0)
            kinds = {}
            for h in ml.history():
                kinds[h["solve"]] = kinds.get(h["solve"], 0) + 1
            fl = ml.predict(Xq).cpu().numpy()
            return dict(fit_s=a0.elapsed_time(a1) / 1e3, newton_steps=ml.info()["newton_steps"],
                        steps_factor=kinds.get(1, 0), steps_reuse=kinds.get(2, 0),
                        steps_lowrank=kinds.get(3, 0), profile=pl,
                        max_decision_diff=float(np.max(np.abs(fl - f.cpu().numpy())
                                                       / np.maximum(1.0, np.abs(f.cpu().numpy())))))
        lowrank = _leg(lowrank_leg)

    # the same fit with the Newton system factored in FP64 (the precision the
    # method's description names; the default factors in FP32 and refines in
    # FP64): fit time, steps and agreement of the decision values
    fp64_factor = None
    if args.fp64_factor:
        def fp64_leg():
            lib.spsvm_profile_enable(1)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            m64 = sp.spsvm_fit(X, y, p.gamma, p.lam, J, 1e-6, workspace=None, newton_solver="fp64",
                               **opts)
            a1.record(stream)
            torch.cuda.synchronize()
            pl = {}
            for k, name in enumerate(SLOTS):
                if name not in ("cholesky", "solve"):
                    continue
                nm, L_, t_, w_ = C.c_char_p(), C.c_int64(), C.c_double(), C.c_double()
                lib.spsvm_profile_read(k, C.byref(nm), C.byref(L_), C.byref(t_), C.byref(w_))
                pl[name] = dict(launches=L_.value, ms=t_.value)
            lib.spsvm_profile_enable(0)
            f64 = m64.predict(Xq).cpu().numpy()
            fr = f.cpu().numpy()
            return dict(fit_s=a0.elapsed_time(a1) / 1e3, newton_steps=m64.info()["newton_steps"],
                        status=m64.status, profile=pl,
                        max_decision_diff=float(np.max(np.abs(f64 - fr) / np.maximum(1.0, np.abs(fr)))))
        fp64_factor = _leg(fp64_leg)

    # FP32 form on the same workload (one fit), for the "vs FP32 form" leg
    fp32_form = None
    if args.fp32_form and prec != "fp32":
        del work
        torch.cuda.empty_cache()

        def fp32_leg():
            o32, _ = sp.make_options(**dict(opts, precision="fp32"))
            w32 = torch.empty(lib.spsvm_fit_workspace_bytes(n, d, J, C.byref(o32)), dtype=torch.uint8,
                              device="cuda")
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            m32 = sp.spsvm_fit(X, y, p.gamma, p.lam, J, 1e-6, workspace=w32,
                               **dict(opts, precision="fp32"))
            a1.record(stream)
            torch.cuda.synchronize()
            f32 = sp.spsvm_predict(m32, Xq).cpu().numpy()
            fb = f.cpu().numpy()
            return dict(fit_s=a0.elapsed_time(a1) / 1e3,
                        label_agreement_with_bf16split=float(np.mean(np.sign(fb) == np.sign(f32))),
                        newton_steps=m32.info()["newton_steps"])

        fp32_form = _leg(fp32_leg)
        torch.cuda.empty_cache()

    # roofline for the dominant kernel of the step
    peaks, src = _peaks()
    dom = max(("gram", "cholesky", "kernel_block", "compact", "gemv", "outputs", "solve", "score",
               "decision", "line_search"), key=lambda k: prof[k]["ms"])
    pr = prof[dom]
    per_launch_ms = pr["ms"] / max(1, pr["launches"])
    per_launch_work = pr["work"] / max(1, pr["launches"])
    # FP32 SIMT rate from the unit counts: SMs x 128 FP32 lanes x 2 flops x
    # the maximum SM clock (sampled; 2,070 MHz when unsampled)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_simt = sms * 128 * 2 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    note = None
    if dom in ("gram", "kernel_block", "score", "decision") and prec == "bf16split":
        # the library counts the plane products of the form in its work
        # (six for the kernel block and the score, four for the Gram matrix)
        bound, unit = "tensor", "TFLOP/s"
        achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e12
        peak = peaks["bf16_tflops_sustained"]
    elif dom in ("gram", "kernel_block", "score", "decision"):
        bound, unit = "alu", "TFLOP/s"
        achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e12
        peak = fp32_simt
    elif dom == "cholesky":
        # |J|^3/3 flops per factorisation of the Newton matrix, done in FP32
        # (FP64 iterative refinement follows in the solve): against the FP32
        # SIMT rate from unit counts and the maximum clock
        bound, unit = "alu", "TFLOP/s"
        achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e12
        peak = fp32_simt
        note = "FP32 factor of the Newton matrix (mixed solve); peak = FP32 SIMT rate derived from unit counts and clock"
    elif dom == "solve":
        # 8 |J|^2 flops per solve (about two refinement steps of two FP32
        # triangular solves and one FP64 residual): chains of 64-row blocks,
        # against the FP32 SIMT rate
        bound, unit = "alu", "TFLOP/s"
        achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e12
        peak = fp32_simt
        note = "refinement of the Newton solve (FP32 triangular solves, FP64 residuals); latency-bound chains; peak = FP32 SIMT rate"
    else:
        bound, unit = "hbm", "GB/s"
        achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
    # DRAM traffic per launch, measured with ncu on the GEMV at n = 100,000
    # (GEMV_TRAFFIC_RATIO x its algorithmic bytes), scaled to this launch size
    traffic = per_launch_work * GEMV_TRAFFIC_RATIO if dom == "gemv" and GEMV_TRAFFIC_RATIO else None
    roofline = dict(kernel=dom, bound=bound, achieved=achieved, peak=peak, unit=unit,
                    frac=achieved / peak, traffic=traffic,
                    peak_source=src if bound in ("hbm", "tensor") else "derived",
                    launches=pr["launches"], ms_per_launch=per_launch_ms)
    if note:
        roofline["note"] = note

    gram_stress = _leg(gram_stress_leg, sp, torch, lib) if args.gram_stress else None
    batched = _leg(batched_leg, sp, torch) if args.batched else None
    ovo = _leg(ovo_leg, sp, torch) if args.ovo else None
    exact = _leg(exact_score_leg, sp, torch) if args.exact_score else None
    serve = (_leg(serve_leg, sp, requests=args.serve_requests, workers=args.serve_workers)
             if args.serve_requests > 0 else None)

    line = dict(metric=METRIC, value=ms / 1e3, unit="s", n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=False, scaling="weak",
                vs_baseline=None,
                dtype=("bf16split" if prec == "bf16split" else "f32") + " kernel/Gram, f32 factor + f64 refinement",
                data="synthetic",
                config=dict(WORKLOAD, precision=prec, l2="inputs larger than L2 (no flush)",
                            step="fit + predict(100k queries)", parallelism=f"replicas{ws}"),
                e2e=dict(value=e2e_ms / 1e3, unit="s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                gpu_launches=int(launches // max(1, args.steps)),
                clocks=clocks, roofline=roofline,
                kernel_block=dict(ms=kb_ms, tflops=kb_tflops, n=n, basis=J, d=d),
                fit=dict(newton_steps=info["newton_steps"], rounds=info["rounds"],
                         objective=info["objective"], status=info["status"]),
                profile={k: v for k, v in prof.items() if v["launches"]},
                fp32_form=fp32_form, lowrank=lowrank, fp64_factor=fp64_factor, growth_stop=growth,
                gram_stress=gram_stress,
                batched=batched, ovo=ovo,
                exact_score=exact, serve=serve)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline_run(steps=1)
        line["cpu_baseline"] = dict(value=cb["sample_seconds"][0], unit="s", cores=cb["nproc"],
                                    kind="oracle", sample=cb["sample"],
                                    blas_threads=cb["blas_threads"], cpu_model=cb["cpu_model"],
                                    points=cb["points"], exponent_n=cb["exponent_n"],
                                    exponent_basis=cb["exponent_basis"],
                                    full_size_estimate_s=cb["full_size_estimate_s"],
                                    gpu_same_sample_s=_leg(gpu_sample_fit_seconds, sp, torch))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16split", choices=["bf16split", "fp32"])
    ap.add_argument("--n", type=int, default=500_000)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--basis", type=int, default=4096)
    ap.add_argument("--queries", type=int, default=100_000)
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end steps (0: the same count as the device-timed steps)")
    ap.add_argument("--fp32-form", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", type=int, default=1)
    ap.add_argument("--serve-requests", type=int, default=100)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--ovo", type=int, default=1, help="one-vs-one leg (10 classes, 45 pairs)")
    ap.add_argument("--exact-score", type=int, default=1,
                    help="heuristic vs exact one-dimensional selection score leg")
    ap.add_argument("--gram-stress", type=int, default=1,
                    help="a fit on an overlapping mixture where the Gram matrix carries real work")
    ap.add_argument("--fp64-factor", type=int, default=1,
                    help="leg: the same fit with the Newton system factored in FP64")
    ap.add_argument("--lowrank", type=int, default=1,
                    help="one fit with the low-rank correction of the Newton factor")
    ap.add_argument("--growth", type=int, default=1,
                    help="report the growth stop at epsilon = 5e-6 and accuracy vs |J|")
    ap.add_argument("--micro", choices=["cholesky", "kblock", "gram"], default=None,
                    help="time one hot-path step alone instead of the whole fit")
    ap.add_argument("--sizes", default="512,1024,2048,4096")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.e2e_steps <= 0:
        args.e2e_steps = args.steps
    if args.impl == "reference":
        return run_reference(args)
    if args.micro == "kblock":
        return run_micro_kblock(args)
    if args.micro == "gram":
        return run_micro_gram(args)
    if args.micro:
        return run_micro(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
