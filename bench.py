"""Benchmark: seconds to relative residual 1e-8 for two-level PCG on GB300.

One step = one pass of the whole hot path over the workload: setup (k-means++
clustering, coarse Gram, Cholesky factor, smoother) at the first lambda, then
for every lambda of the workload the coarse factor at that lambda and a solve
of (X^T X + lambda I) w = X^T y to ||r|| <= 1e-8 ||X^T y||.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun (N > 1) every rank runs an
independent replica of the workload on its own GPU ("replicas only": one
solve does not shard), value = the slowest rank's seconds per step.
--impl reference times the FP64 CPU oracle on the host cores instead, each
step a bounded sample of the same workload extrapolated to the full step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s to rel. residual 1e-8: batched/learned vs plain two-level PCG, same GB300"
WORKLOAD = "zipf_200000x100000"
TOL = 1e-8
LEADER_TOL2 = (1000.0,)   # the leader-follower section's squared tolerance(s)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-parity", action="store_true",
                    help="skip the oracle's exact solutions of the workload (error of each solve)")
    ap.add_argument("--no-eigen", action="store_true",
                    help="skip the section comparing the eigendecomposition coarse solve")
    ap.add_argument("--no-bayes", action="store_true",
                    help="skip the Gibbs-sampling (rr_bayes) section")
    ap.add_argument("--only-bayes", action="store_true",
                    help="only the Gibbs-sampling section")
    ap.add_argument("--no-leader", action="store_true",
                    help="skip the leader-follower section")
    ap.add_argument("--many-workload", default="uneven_12_dense4",
                    help="the independent-problem set of --only many (uneven_28_dense4: the "
                         "specified 28 + 4 problems, minutes of host generation)")
    ap.add_argument("--only-leader", action="store_true",
                    help="only the leader-follower section (--leader-tol2 list)")
    ap.add_argument("--leader-tol2", default="",
                    help="comma-separated squared tolerances of the leader-follower section")
    ap.add_argument("--only-eigen", action="store_true",
                    help="run the eigendecomposition section alone (profiling runs)")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the small FP64 configuration (2,000 x 1,000, us per iteration)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched section (64 targets x 8 weights over the same X)")
    ap.add_argument("--no-many", action="store_true",
                    help="skip the section of uneven independent problems in one graph")
    ap.add_argument("--no-tlfcg", action="store_true",
                    help="skip the section solving the same systems with the paper's TLFCG")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned coarse correction section (harvest, training, solves)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="host-issued loops instead of CUDA graphs (every kernel visible to a profiler)")
    ap.add_argument("--gather", default="auto", choices=["auto", "lanes", "staged", "lanes-staged"],
                    help="FP32 gather kernel (auto: timed per pass at setup; the others force one; "
                         "lanes-staged: lanes for X, staged for X^T)")
    ap.add_argument("--only", choices=["batched", "many", "learned", "dense"],
                    help="run one extra section alone and print it (profiling runs)")
    ap.add_argument("--batch-targets", type=int, default=64,
                    help="targets of the batched section (64: the zipf_200000x100000_64x8 workload)")
    ap.add_argument("--pairs", type=int, default=100_000,
                    help="training pairs of the learned section (100,000 by default)")
    ap.add_argument("--profile-step", action="store_true",
                    help="one untimed step and nothing else (for a profiler's launch list)")
    ap.add_argument("--roofline-only", action="store_true",
                    help="one setup, then only the operator-apply kernel timings (profiling runs)")
    ap.add_argument("--profile-apply", type=int, default=0, metavar="K",
                    help="one setup and three warm-up applies, then K operator applies between "
                         "cudaProfilerStart/Stop (ncu --profile-from-start off); nothing timed")
    ap.add_argument("--split-head", type=int, default=0,
                    help="head columns of the FP32 operator's split form (0: automatic, -1: none)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="mixed: FP32 operator inside CG + FP64 refinement; fp64: FP64 throughout")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def slowest_over_ranks(ms, world, device=None):
    """The largest of the ranks' values (the slowest replica sets a step's time);
    the value itself on one rank. Needs the process group when world > 1."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline inputs

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profiled_traffic(kernel, workload):
    """dram read+write bytes per launch recorded by an ncu capture in profiles/."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null") else float(v)
    except OSError:
        pass
    return None


# ---------------------------------------------------------------- parity leg

def _parity_worker(spec, k, seed, jobs, out_path, threads):
    """Runs in a spawned process: the oracle's clustering, then the exact
    solution of every (lambda, y) job (the oracle's PCG to 1e-12, one process
    each), saved to out_path."""
    sys.path.insert(0, ROOT)
    from oracle import reference
    _, raw, iters = reference.oracle_labels(spec, k, seed, threads=threads)
    res = reference.exact_solutions(spec, raw, list(jobs), snap_tols=(TOL,),
                                    processes=len(jobs))
    np.savez(out_path, w_ref=np.stack([r[0] for r in res]),
             w_orc=np.stack([r[1][TOL] for r in res]),
             iters=np.array([r[2] for r in res]), rel=np.array([r[3] for r in res]),
             kmeans_iters=iters)


# systems of the batched workload checked against the oracle: (weight index,
# target index) of zipf_200000x100000_64x8
BATCH_SAMPLES = ((0, 0), (7, 63))


def start_parity(X, y, p, tmpdir, batch=True):
    """Starts the oracle's exact solutions in the background (before any GPU
    work is timed; the process is spawned, so it shares nothing with the CUDA
    context): the step's systems, then (batch) the sampled batched systems.
    Returns (process, output path)."""
    import multiprocessing as mp
    from gen import synth
    spec = (X.n_rows, X.n_cols, p["density"], p["s"], p["seed"])
    path = os.path.join(tmpdir, "parity.npz")
    threads = max(1, (os.cpu_count() or 4) // 2 - 1)
    jobs = [(lam, y) for lam in p["lambdas"]]
    if batch:
        pb = synth.BATCH_WORKLOADS["zipf_200000x100000_64x8"]
        for l, j in BATCH_SAMPLES:
            yj, _ = synth.ridge_targets_many(X, [pb["target_seeds"][j]])
            jobs.append((float(pb["lambdas"][l]), yj[0]))
    proc = mp.get_context("spawn").Process(
        target=_parity_worker, args=(spec, p["k"], p["seed"], jobs, path, threads),
        daemon=False)
    proc.start()
    return proc, path


# the factor of the solution bar: at relative residual 1e-8 the error of a
# correct solve varies with the method by up to about 11x the oracle PCG's own
# (measured over 72 small systems, the mixed-precision refinement form the
# widest); the bar takes about twice that (the tests use the same factor)
SOLUTION_SPREAD = 25.0


def finish_parity(proc, path, W, lams, timeout_s=900, W_batch=None):
    """||w - w_ref|| / ||w_ref|| of the timed step's solutions (and of the
    sampled batched systems, when given), with the oracle's own error at the
    same tolerance for context. Returns (step parity, batched parity)."""
    proc.join(timeout_s)
    if proc.is_alive() or not os.path.exists(path):
        if proc.is_alive():
            proc.terminate()
        return {"error": "the oracle's reference solve did not finish"}, None
    d = np.load(path)

    def compare(ws, idx):
        o = {"err_vs_oracle": [], "oracle_err_at_tol": [], "bar": [], "within_bar": []}
        for w, j in zip(ws, idx):
            wr = d["w_ref"][j]
            e = float(np.linalg.norm(w - wr) / np.linalg.norm(wr))
            eo = float(np.linalg.norm(d["w_orc"][j] - wr) / np.linalg.norm(wr))
            bar = max(1e-6, SOLUTION_SPREAD * eo)
            o["err_vs_oracle"].append(e)
            o["oracle_err_at_tol"].append(eo)
            o["bar"].append(bar)
            o["within_bar"].append(bool(e <= bar))
        return o

    out = {"reference": "oracle two-level PCG (its own k-means++ clustering) to relative residual "
                        "1e-12", "tol": TOL, "lambdas": list(lams)}
    out.update(compare(W, range(len(lams))))
    out["oracle_ref_iters"] = [int(v) for v in d["iters"][:len(lams)]]
    out["oracle_kmeans_iters"] = int(d["kmeans_iters"])
    bout = None
    if W_batch is not None and len(d["w_ref"]) >= len(lams) + len(BATCH_SAMPLES):
        bout = {"systems": [list(s) for s in BATCH_SAMPLES],
                "note": "(weight index, target index) of the batched workload"}
        bout.update(compare(W_batch, range(len(lams), len(lams) + len(BATCH_SAMPLES))))
    return out, bout


def measure_small_fp64(rr, dev):
    """The small plain FP64 configuration (2,000 x 1,000, 1%, k = 50,
    lambda = 1e-2, seed 0): latency-bound, so reported as microseconds per
    PCG iteration, with the error against a dense solve."""
    import torch
    from gen import synth
    from oracle import sparse as osp
    X, y, _, p = synth.workload("zipf_2000x1000")
    lam = p["lambdas"][0]
    h = rr.rr_setup(X.row_ptr, X.col_idx, X.n_rows, X.n_cols, lam, p["k"], seed=p["seed"])
    yd = torch.as_tensor(y, device=dev)
    w = torch.empty(X.n_cols, dtype=torch.float64, device=dev)
    for _ in range(3):
        info = rr.rr_solve(h, yd, w, tol=TOL)
    ms = []
    for _ in range(5):
        info = rr.rr_solve(h, yd, w, tol=TOL)
        ms.append(info["solve_ms"])
    M = osp.from_csr(X.n_rows, X.n_cols, X.row_ptr, X.col_idx)
    wr = np.linalg.solve(osp.dense_A(M, lam), osp.rhs(M, y))
    err = float(np.linalg.norm(w.cpu().numpy() - wr) / np.linalg.norm(wr))
    rr.rr_free(h)
    med = statistics.median(ms)
    return {"workload": "zipf_2000x1000", "precision": "fp64", "setup_ms": round(info["setup_ms"], 2),
            "solve_ms": round(med, 3), "iters": info["iters"],
            "us_per_iter": round(1000 * med / max(1, info["iters"]), 2),
            "err_vs_dense_solve": err, "true_rel_res": info["true_rel_res"],
            "note": "latency bound (0.5 MB per iteration, L2 resident): no HBM fraction"}


# ---------------------------------------------------------------- our arm

def measure_roofline(rr, row_ptr, col_idx, N, F, nnz, k, lams, opts, dev, stream, workload):
    """Operator-apply kernels timed alone with CUDA events on the library's stream."""
    import torch
    h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], k, **opts)
    v = torch.randn(F, dtype=torch.float64, device=dev)
    u = torch.empty(N, dtype=torch.float64, device=dev)
    z = torch.empty(F, dtype=torch.float64, device=dev)
    reps = 20
    kern = {}
    for name, fn in (("X_v", lambda: rr.rr_matvec(h, v, u)),
                     ("Xt_u", lambda: rr.rr_rhs(h, u, z)),
                     ("A_v", lambda: rr.rr_apply(h, v, z))):
        for _ in range(3):
            fn()
        es = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        for i in range(reps):
            es[2 * i].record(stream)
            fn()
            es[2 * i + 1].record(stream)
        torch.cuda.synchronize(dev)
        kern[name] = statistics.mean(es[2 * i].elapsed_time(es[2 * i + 1]) for i in range(reps))
    rr.rr_free(h)
    # algorithmic bytes per call: one int32 index per nonzero per pass, the
    # pointer array of the pass, each vector read or written once
    algo = {
        "X_v": 4 * nnz + 8 * (N + 1) + 8 * F + 8 * N,
        "Xt_u": 4 * nnz + 8 * (F + 1) + 8 * N + 8 * F,
        "A_v": 8 * nnz + 8 * (N + 1) + 8 * (F + 1) + 8 * F + 16 * N + 8 * F + 8 * F,
    }
    dom = "A_v"
    peak, peak_kind = peaks()
    achieved = algo[dom] / (kern[dom] * 1e-3) / 1e9
    return {"bound": "hbm",
            "kernel": "operator apply, split form (tail gathers x2, k_split_rows, k_split_epilogue)"
                      if opts.get("precision") == rr.RR_PREC_MIXED else
                      "operator apply (k_sliced_gather x2 + k_sliced_epilogue)",
            "achieved": round(achieved, 1), "peak": peak,
            "peak_kind": f"{peak_kind} (burst copy)", "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": profiled_traffic("operator_apply_split" if opts.get("precision") ==
                                        rr.RR_PREC_MIXED else "operator_apply", workload),
            "algorithmic_bytes": algo[dom], "launch_ms": round(kern[dom], 4),
            "parts": {n: {"ms": round(t, 4), "achieved_gbs": round(algo[n] / (t * 1e-3) / 1e9, 1)}
                      for n, t in kern.items() if n != dom}}


def measure_batched(rr, X, row_ptr, col_idx, k, opts, dev, stream, world, n_targets=64):
    """Many targets and weights over the same X in one rr_solve_batch (the
    batched form), against the plain two-level PCG solving a sample of the same
    systems one at a time on the same GPU. One warm-up, then one timed run of
    setup + batch solve (CUDA events on the library's stream)."""
    import torch
    from gen import synth
    name = "zipf_200000x100000_64x8"
    pb = synth.BATCH_WORKLOADS[name]
    seeds, lams = pb["target_seeds"][:n_targets], list(pb["lambdas"])
    if n_targets != len(pb["target_seeds"]):
        name += f" (first {n_targets} targets)"
    Y, _ = synth.ridge_targets_many(X, seeds)
    N, F = X.n_rows, X.n_cols
    Yd = torch.as_tensor(Y, device=dev)
    Wb = torch.empty((len(lams), len(seeds), F), dtype=torch.float64, device=dev)

    def run():
        h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], k, **opts)
        out = rr.rr_solve_batch(h, Yd, lams, Wb, tol=TOL)
        return h, out

    h, out = run()
    rr.rr_free(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    h, out = run()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_batch = e0.elapsed_time(e1) / 1000.0
    infos = [i for row in out["infos"] for i in row]
    assert out["status"] == "RR_OK" and max(i["true_rel_res"] for i in infos) <= TOL
    # the plain two-level PCG on every system, one solve after the other on the
    # same handle (the same setup; rr_set_lambda per weight), timed with events
    w = torch.empty(F, dtype=torch.float64, device=dev)
    plain_ms, e2 = [], [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for lam in lams:
        rr.rr_set_lambda(h, lam)
        e2[0].record(stream)
        for j in range(len(seeds)):
            inf = rr.rr_solve(h, Yd[j], w, tol=TOL)
            assert inf["status"] == "RR_OK"
        e2[1].record(stream)
        torch.cuda.synchronize(dev)
        plain_ms.append(e2[0].elapsed_time(e2[1]))
    n_sys = len(infos)
    setup_s = infos[0]["setup_ms"] / 1000.0
    t_plain = setup_s + sum(plain_ms) / 1000.0
    # the operator apply of the whole batch (both FP32 passes over every slab,
    # the autotuned variant), against its algorithmic bytes: the two index
    # streams once per slab, V read, U written and read, Z written; and the
    # row-segment gathers (every index fetches 4 bytes per system of its slab)
    q = rr.rr_query_batch(h)
    ld = -(-n_sys // 64) * 64
    nnz = X.nnz
    slabs = -(-ld // q["slab_width"])
    alg = slabs * 8 * nnz + 4 * F * ld + 8 * N * ld + 4 * F * ld
    peak, peak_kind = peaks()
    sec = q["apply_ms"] * 1e-3
    batched_roofline = {
        "bound": "l2 (row-segment gathers)", "kernel": "batched SpMM apply (k_bspmm x2)",
        "slab_width": q["slab_width"], "unroll": q["unroll"], "apply_ms": round(q["apply_ms"], 4),
        "algorithmic_bytes": alg, "achieved": round(alg / sec / 1e9, 1), "unit": "GB/s",
        "peak": peak, "peak_kind": f"{peak_kind} (burst copy)",
        "frac": round(alg / sec / 1e9 / peak, 4),
        "l2_gather_bytes": 2 * nnz * ld * 4, "l2_gather_tbs": round(2 * nnz * ld * 4 / sec / 1e12, 2),
        "per_system_apply_us": round(q["apply_ms"] * 1e3 / n_sys, 2)}
    rr.rr_free(h)
    its = sorted(i["iters"] for i in infos)
    samples = [Wb[l, j].cpu().numpy() for l, j in BATCH_SAMPLES if j < len(seeds)]
    return {"workload": name, "systems": n_sys, "targets": len(seeds), "lambdas": lams,
            "_samples": samples if len(samples) == len(BATCH_SAMPLES) else None,
            "value": round(t_batch, 4), "unit": "s", "s_per_system": round(t_batch / n_sys, 6),
            "setup_s": round(setup_s, 4), "solve_s": round(infos[0]["solve_ms"] / 1000.0, 4),
            "iters_min_median_max": [its[0], its[len(its) // 2], its[-1]],
            "restarts_max": max(i["restarts"] for i in infos),
            "true_rel_res_max": max(i["true_rel_res"] for i in infos),
            "plain_solve_ms_per_lambda": [round(t, 2) for t in plain_ms],
            "plain_s": round(t_plain, 3),
            "speedup_vs_plain": round(t_plain / t_batch, 2),
            "roofline": batched_roofline,
            "note": "plain = one setup + rr_solve of every system one after the other"}


def measure_eigen(rr, row_ptr, col_idx, N, F, k, lams, opts, dev, stream, y_dev):
    """The coarse solve by eigendecomposition (RR_COARSE_EIGEN) against the
    Cholesky form on the same workload: the setup's coarse-factor phase (the
    Jacobi eigendecomposition once, against one Cholesky factorisation), the
    cost of one lambda change (rr_set_lambda, the 8 weights of the batched
    workload, CUDA events) and a solve at each lambda of the step."""
    import torch
    from gen import synth
    out = {}
    weights = list(synth.BATCH_WORKLOADS["zipf_200000x100000_64x8"]["lambdas"])
    w = torch.empty(F, dtype=torch.float64, device=dev)
    for name, coarse in (("cholesky", rr.RR_COARSE_CHOLESKY), ("eigen", rr.RR_COARSE_EIGEN)):
        h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], k, **dict(opts, coarse=coarse))
        info = rr.rr_solve(h, y_dev, w, tol=TOL)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for lam in weights:
            rr.rr_set_lambda(h, lam)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        iters = []
        for lam in lams:
            rr.rr_set_lambda(h, lam)
            inf = rr.rr_solve(h, y_dev, w, tol=TOL)
            assert inf["status"] == "RR_OK" and inf["true_rel_res"] <= TOL
            iters.append(inf["iters"])
        out[name] = {"coarse_factor_phase_ms": round(info["setup_phase_ms"][6], 2),
                     "setup_ms": round(info["setup_ms"], 2),
                     "set_lambda_ms": round(ev[0].elapsed_time(ev[1]) / len(weights), 3),
                     "iters": iters}
        if coarse == rr.RR_COARSE_EIGEN:
            out[name]["jacobi_sweeps"] = rr.rr_get_eigen(h)[2]
        rr.rr_free(h)
    ch, eg = out["cholesky"], out["eigen"]
    extra = eg["coarse_factor_phase_ms"] - ch["coarse_factor_phase_ms"]
    saved = ch["set_lambda_ms"] - eg["set_lambda_ms"]
    out["break_even_lambdas"] = round(extra / saved, 1) if saved > 0 else None
    return out


def measure_bayes(rr, row_ptr, col_idx, N, F, k, lam, opts, dev, y_dev, n_samples=8, burnin=2):
    """Bayesian ridge regression by Gibbs sampling with noise injection
    (rr_bayes): every sample solves the system at a new lambda / tau, so the
    coarse solve is rebuilt each time; Cholesky (a factorisation per sample)
    against the eigendecomposition (two mat-vec scalings per sample). Wall
    time of the synchronous call over n_samples, per sample."""
    import time
    import torch
    out = {"n_samples": n_samples, "burnin": burnin,
           "prior": {"alpha": 1.0, "beta": 1.0, "a_tau": 1.0, "b_tau": 1.0}, "tol": TOL}
    wm = torch.empty(F, dtype=torch.float64, device=dev)
    for name, coarse in (("cholesky", rr.RR_COARSE_CHOLESKY), ("eigen", rr.RR_COARSE_EIGEN)):
        h = rr.rr_setup(row_ptr, col_idx, N, F, lam, k, **dict(opts, coarse=coarse))
        rr.rr_bayes(h, y_dev, 2, 0, wm, tol=TOL, seed=1)          # warm-up
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        lams, taus, iters = rr.rr_bayes(h, y_dev, n_samples, burnin, wm, tol=TOL, seed=2)
        torch.cuda.synchronize(dev)
        ms = (time.perf_counter() - t0) * 1e3
        out[name] = {"ms_per_sample": round(ms / n_samples, 2), "iters": [int(i) for i in iters],
                     "lambda_last": float(lams[-1]), "tau_last": float(taus[-1])}
        rr.rr_free(h)
    out["speedup_eigen"] = round(out["cholesky"]["ms_per_sample"] /
                                 max(1e-9, out["eigen"]["ms_per_sample"]), 3)
    return out


def measure_leader(rr, row_ptr, col_idx, N, F, lams, opts, dev, y_dev, tol2s, cap=16384,
                   tlfcg=True, kmeans_same_k=False):
    """Leader-follower clustering (Algorithm 1, RR_CLUSTER_LEADER) in place of
    k-means++ on the step's matrix: for each squared tolerance, the number of
    leaders (the coarse size F_C), the clustering's time, the setup, and the
    two-level PCG (and, with tlfcg, the paper's TLFCG) at each lambda of the
    step, against the k-means++ numbers of the timed step."""
    import torch
    out = {"tol2": [], "cap": cap}
    w = torch.empty(F, dtype=torch.float64, device=dev)
    for tol2 in tol2s:
        row = {"tol2": tol2}
        try:
            h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], cap,
                            **dict(opts, clustering=rr.RR_CLUSTER_LEADER, lf_tol2=tol2))
        except rr.RRError as e:
            row["error"] = str(e)[:120]
            out["tol2"].append(row)
            continue
        row["k_eff"] = rr.rr_query(h)["k_eff"]
        row["pcg_iters"], row["pcg_solve_ms"] = [], []
        info = None
        for j, lam in enumerate(lams):
            if j:
                rr.rr_set_lambda(h, lam)
            info = rr.rr_solve(h, y_dev, w, tol=TOL)
            assert info["status"] == "RR_OK" and info["true_rel_res"] <= TOL
            row["pcg_iters"].append(info["iters"])
            row["pcg_solve_ms"].append(round(info["solve_ms"], 2))
        row["setup_ms"] = round(info["setup_ms"], 2)
        row["cluster_ms"] = round(info["setup_phase_ms"][2] + info["setup_phase_ms"][3], 2)
        rr.rr_free(h)
        if tlfcg:
            h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], cap,
                            **dict(opts, clustering=rr.RR_CLUSTER_LEADER, lf_tol2=tol2,
                                   solver=rr.RR_SOLVER_TLFCG))
            inf = rr.rr_solve(h, y_dev, w, tol=TOL)
            assert inf["status"] == "RR_OK" and inf["true_rel_res"] <= TOL
            row["tlfcg_iters_lam0"] = inf["iters"]
            row["tlfcg_solve_ms_lam0"] = round(inf["solve_ms"], 2)
            rr.rr_free(h)
        if kmeans_same_k:
            # k-means++ into as many clusters as there are leaders: the coarse
            # size and the clustering method told apart
            km = {"k": row["k_eff"]}
            h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], row["k_eff"], **opts)
            inf = rr.rr_solve(h, y_dev, w, tol=TOL)
            km["pcg_iters_lam0"] = inf["iters"]
            km["setup_ms"] = round(inf["setup_ms"], 2)
            km["cluster_ms"] = round(inf["setup_phase_ms"][2] + inf["setup_phase_ms"][3], 2)
            rr.rr_free(h)
            h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], row["k_eff"],
                            **dict(opts, solver=rr.RR_SOLVER_TLFCG))
            inf = rr.rr_solve(h, y_dev, w, tol=TOL)
            km["tlfcg_iters_lam0"] = inf["iters"]
            rr.rr_free(h)
            row["kmeans_same_k"] = km
        out["tol2"].append(row)
    return out


def measure_tlfcg(rr, row_ptr, col_idx, N, F, k, lams, opts, y_dev):
    """The same systems (each lambda, same target, same clustering) solved by the
    paper's TLFCG: flexible CG whose preconditioner is two CG rougher steps and the
    coarse correction; against the plain two-level PCG, both one weight after the
    other on one handle (rr_set_lambda)."""
    import torch
    w = torch.empty(F, dtype=torch.float64, device=y_dev.device)
    runs = {}
    for name, solver in (("tlfcg", rr.RR_SOLVER_TLFCG), ("pcg", rr.RR_SOLVER_TWOLEVEL)):
        h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], k, **dict(opts, solver=solver))
        runs[name] = []
        for j, lam in enumerate(lams):
            if j:
                rr.rr_set_lambda(h, lam)
            runs[name].append(rr.rr_solve(h, y_dev, w, tol=TOL))
        rr.rr_free(h)
    out = {"method": "FCG(1), preconditioner: 2 CG steps on A z = r, then the coarse correction",
           "iters": [i["iters"] for i in runs["tlfcg"]],
           "solve_ms": [round(i["solve_ms"], 2) for i in runs["tlfcg"]],
           "true_rel_res": [i["true_rel_res"] for i in runs["tlfcg"]]}
    out["pcg_iters"] = [i["iters"] for i in runs["pcg"]]
    out["pcg_solve_ms"] = [round(i["solve_ms"], 2) for i in runs["pcg"]]
    out["speedup_vs_pcg"] = round(sum(out["pcg_solve_ms"]) / max(1e-9, sum(out["solve_ms"])), 3)
    return out


def measure_dense_apply(rr, h, n, f, dev, stream, reps=20):
    """The dense operator apply X^T X v + lambda v on a dense handle, in the
    handle's precision (the one the CG iterations use): X is read once (4 n f
    bytes) plus v and the result (16 f bytes); X (800 MB at 50,000 x 4,000) is
    larger than L2."""
    import torch
    v = torch.randn(f, dtype=torch.float64, device=dev)
    o = torch.empty_like(v)
    for _ in range(3):
        rr.rr_apply(h, v, o)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    for _ in range(reps):
        rr.rr_apply(h, v, o)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    ms = ev[0].elapsed_time(ev[1]) / reps
    alg = 4 * n * f + 16 * f
    return {"n": n, "d": f, "ms": round(ms, 4), "algorithmic_bytes": alg,
            "achieved_gbs": round(alg / ms / 1e6, 1)}


def measure_dense_only(rr, dev, stream, opts):
    """One dense problem of the many-problem workload (50,000 x 4,000 AR(1),
    rho = 0.9, seed 12, k = 40): setup, then the dense operator apply."""
    import torch
    from gen import synth
    p = next(q for q in synth.many_params("uneven_12_dense4") if q.get("dense"))
    n, f = p["n"], p["d"]
    X = synth.dense_ar1(n, f, p["rho"], p["seed"])
    o = {key: v for key, v in opts.items() if key not in ("gram", "gather", "seed", "split_head")}
    h = rr.rr_setup_dense(torch.as_tensor(X, device=dev), p["lam"], p["k"], seed=p["seed"], **o)
    out = measure_dense_apply(rr, h, n, f, dev, stream)
    rr.rr_free(h)
    return out


def measure_many(rr, dev, stream, opts, name="uneven_12_dense4"):
    """Independent problems of uneven sizes: rr_solve_many (all PCG loops in one
    graph) against rr_solve one problem after the other, same handles (setups
    excluded from both; they are reported apart). The problems are generated
    one at a time and only their handles kept. The binary problem with the
    fewest nonzeros is checked against the oracle's exact solution (its own
    clustering, PCG to 1e-12, in a spawned process that runs meanwhile)."""
    import multiprocessing as mp
    import torch
    from gen import synth
    params = synth.many_params(name)
    binary = [q for q in params if not q.get("dense")]
    q0 = min(binary, key=lambda q: q["n"] * q["d"] * q["density"])
    X0, y0 = synth.many_problem(q0)
    tmpdir = tempfile.mkdtemp(prefix="rr_many_")
    ppath = os.path.join(tmpdir, "parity.npz")
    pproc = mp.get_context("spawn").Process(
        target=_parity_worker,
        args=((q0["n"], q0["d"], q0["density"], 1.1, q0["seed"]), q0["k"], q0["seed"],
              [(q0["lam"], y0)], ppath, max(1, (os.cpu_count() or 4) // 2 - 1)), daemon=False)
    pproc.start()
    del X0
    probs = []
    hs, ys, ws, setup_ms = [], [], [], []
    t_gen = 0.0
    for p in params:
        t0 = time.time()
        X, y = synth.many_problem(p)
        t_gen += time.time() - t0
        probs.append((X.shape if p.get("dense") else (X.n_rows, X.n_cols, X.nnz), p))
        if p.get("dense"):
            o = {key: v for key, v in opts.items() if key not in ("gram", "gather", "split_head")}
            h = rr.rr_setup_dense(torch.as_tensor(X, device=dev), p["lam"], p["k"],
                                  **dict(o, seed=p["seed"]))
            hs.append(h)
            ys.append(torch.as_tensor(y, device=dev))
            ws.append(torch.empty(X.shape[1], dtype=torch.float64, device=dev))
            continue
        rp = torch.as_tensor(X.row_ptr, device=dev)
        ci = torch.as_tensor(X.col_idx, device=dev)
        h = rr.rr_setup(rp, ci, X.n_rows, X.n_cols, p["lam"], p["k"], **dict(opts, seed=p["seed"]))
        del rp, ci
        hs.append(h)
        ys.append(torch.as_tensor(y, device=dev))
        ws.append(torch.empty(X.n_cols, dtype=torch.float64, device=dev))
        del X
    out = rr.rr_solve_many(hs, ys, ws, tol=TOL, stream=stream)   # warm-up
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize(dev)
    e[0].record(stream)
    out = rr.rr_solve_many(hs, ys, ws, tol=TOL, stream=stream)
    e[1].record(stream)
    torch.cuda.synchronize(dev)
    assert out["status"] == "RR_OK" and max(i["true_rel_res"] for i in out["infos"]) <= TOL
    e[2].record(stream)
    singles = [rr.rr_solve(h, y, w, tol=TOL) for h, y, w in zip(hs, ys, ws)]
    e[3].record(stream)
    torch.cuda.synchronize(dev)
    t_many, t_seq = e[0].elapsed_time(e[1]) / 1e3, e[2].elapsed_time(e[3]) / 1e3
    sizes = [(s[0], s[1], s[0] * s[1]) if p.get("dense") else tuple(s) for s, p in probs]
    dense_apply = None
    for h, (s, p) in zip(hs, probs):
        if p.get("dense"):
            dense_apply = measure_dense_apply(rr, h, s[0], s[1], dev, stream)
            break
    i0 = params.index(q0)
    w0 = ws[i0].cpu().numpy()
    for h in hs:
        rr.rr_free(h)
    pproc.join(900)
    parity = {"error": "the oracle's reference solve did not finish"}
    if not pproc.is_alive() and os.path.exists(ppath):
        d = np.load(ppath)
        wr = d["w_ref"][0]
        err = float(np.linalg.norm(w0 - wr) / np.linalg.norm(wr))
        eo = float(np.linalg.norm(d["w_orc"][0] - wr) / np.linalg.norm(wr))
        parity = {"problem": i0, "n_d": [q0["n"], q0["d"]], "err_vs_oracle": err,
                  "oracle_err_at_tol": eo, "bar": max(1e-6, SOLUTION_SPREAD * eo),
                  "within_bar": bool(err <= max(1e-6, SOLUTION_SPREAD * eo))}
    elif pproc.is_alive():
        pproc.terminate()
    return {"workload": name, "problems": len(probs), "value": round(t_many, 4), "unit": "s",
            "generation_s": round(t_gen, 1), "parity": parity,
            "sequential_s": round(t_seq, 4), "speedup_vs_sequential": round(t_seq / t_many, 2),
            "setup_s_total": round(sum(i["setup_ms"] for i in singles) / 1e3, 3),
            "iters": [i["iters"] for i in out["infos"]],
            "true_rel_res_max": max(i["true_rel_res"] for i in out["infos"]),
            "sizes_n_d_nnz": sizes, "dense_apply": dense_apply}


def measure_learned(rr, X, row_ptr, col_idx, k, opts, dev, stream, n_pairs=100_000,
                    eval_seeds=tuple(range(100, 116)), hidden=512):
    """The learned coarse correction on the 200,000 x 100,000 matrix at
    lambda = 1e-3: pairs harvested from two-level PCG on training targets
    (seeds 1000+, 64 per batch), the network (k -> 512 -> 512 -> k, BF16
    tensor-core training, Adam) trained on the GPU, then held-out targets solved
    by FCG with the learned correction (fallback to the Cholesky coarse solve)
    and by the plain two-level PCG; both to true residual 1e-8."""
    import torch
    from gen import synth
    lam = 1e-3
    N, F = X.n_rows, X.n_cols
    h = rr.rr_setup(row_ptr, col_idx, N, F, lam, k, **opts)
    k_eff = rr.rr_query(h)["k_eff"]
    t0 = time.time()
    Xs, Ts, got, seed0 = [], [], 0, 1000
    u = torch.empty(N, dtype=torch.float64, device=dev)

    def targets(seeds):
        # y = X w* + N(0, 0.1^2) as the generator defines it, X w* by the library's X v
        Y = np.empty((len(seeds), N))
        for j, sd in enumerate(seeds):
            rr.rr_matvec(h, torch.as_tensor(synth.normal(sd, 10, F), device=dev), u)
            Y[j] = u.cpu().numpy() + 0.1 * synth.normal(sd, 11, N)
        return torch.as_tensor(Y, device=dev)

    while got < n_pairs:
        seeds = list(range(seed0, seed0 + 64))
        seed0 += 64
        Yd = targets(seeds)
        Wref = torch.empty((1, 64, F), dtype=torch.float64, device=dev)
        rr.rr_solve_batch(h, Yd, [lam], Wref, tol=1e-10)
        xp, tp = rr.rr_harvest(h, Yd, lam, Wref[0].contiguous(), 1e-8, 400, n_pairs - got, k_eff)
        Xs.append(xp)
        Ts.append(tp)
        got += xp.shape[0]
    Xp, Tp = torch.cat(Xs), torch.cat(Ts)
    t_harvest = time.time() - t0
    params = synth.mlp_init(k_eff, hidden, seed=7)
    net = rr.mlp_create(k_eff, hidden, params, max_batch=512, stream=stream)
    steps = 2000
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = rr.mlp_train(net, Xp, Tp, batch=512, steps=steps, lr=1e-3, seed=3)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_train = e0.elapsed_time(e1) / 1e3
    # the same pairs and steps with the loss weighted by A_c (scaled by its
    # largest diagonal entry): the error of a coarse correction in the energy
    # norm of the coarse space
    Ac, _ = rr.rr_get_coarse(h)
    net_w = rr.mlp_create(k_eff, hidden, params, max_batch=512, stream=stream)
    rr.mlp_set_metric(net_w, Ac / np.abs(np.diag(Ac)).max())
    losses_w = rr.mlp_train(net_w, Xp, Tp, batch=512, steps=steps, lr=1e-3, seed=3)
    w = torch.empty(F, dtype=torch.float64, device=dev)
    rows = []
    for s in eval_seeds:
        yd = targets([s])[0].contiguous()
        a = rr.rr_solve_fcg(h, net, yd, w, tol=TOL)
        b = rr.rr_solve(h, yd, w, tol=TOL)
        c = rr.rr_solve_fcg(h, None, yd, w, tol=TOL)
        d = rr.rr_solve_fcg(h, net_w, yd, w, tol=TOL)
        for inf in (a, b, c, d):
            assert inf["status"] == "RR_OK" and inf["true_rel_res"] <= TOL
        rows.append((a["solve_ms"], a["iters"], a["fallbacks"], b["solve_ms"], b["iters"],
                     c["solve_ms"], c["iters"], d["solve_ms"], d["iters"], d["fallbacks"]))
    r = np.array(rows, dtype=np.float64)
    net.close()
    net_w.close()
    rr.rr_free(h)
    return {"workload": "zipf_200000x100000 lambda=1e-3", "pairs": int(Xp.shape[0]),
            "net": f"{k_eff}-{hidden}-{hidden}-{k_eff} BF16 (tcgen05 training)",
            "harvest_s": round(t_harvest, 2), "train_s": round(t_train, 3),
            "train_steps": steps, "batch": 512,
            "loss_first_last": [float(losses[:20].mean()), float(losses[-20:].mean())],
            "held_out_seeds": len(eval_seeds),
            "learned_fcg_s_mean": round(r[:, 0].mean() / 1e3, 4),
            "learned_fcg_iters_mean": round(r[:, 1].mean(), 1),
            "learned_fallbacks_mean": round(r[:, 2].mean(), 1),
            "plain_pcg_s_mean": round(r[:, 3].mean() / 1e3, 4),
            "plain_pcg_iters_mean": round(r[:, 4].mean(), 1),
            "cholesky_fcg_s_mean": round(r[:, 5].mean() / 1e3, 4),
            "cholesky_fcg_iters_mean": round(r[:, 6].mean(), 1),
            "speedup_vs_plain": round(r[:, 3].mean() / r[:, 0].mean(), 3),
            "ac_weighted_loss": {
                "loss": "0.5/B sum (o - t)^T (A_c / max diag A_c) (o - t)",
                "loss_first_last": [float(losses_w[:20].mean()), float(losses_w[-20:].mean())],
                "learned_fcg_s_mean": round(r[:, 7].mean() / 1e3, 4),
                "learned_fcg_iters_mean": round(r[:, 8].mean(), 1),
                "learned_fallbacks_mean": round(r[:, 9].mean(), 1),
                "fallback_rate": round(r[:, 9].sum() / max(1.0, r[:, 8].sum()), 3),
                "speedup_vs_plain": round(r[:, 3].mean() / r[:, 7].mean(), 3)},
            "fallback_rate": round(r[:, 2].sum() / max(1.0, r[:, 1].sum()), 3)}


def run_ours(args, rank, world, local):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from gen import synth
    from paper_1806_05826_gb300 import rr

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    if args.only == "dense":
        prec = rr.RR_PREC_MIXED if args.precision == "mixed" else rr.RR_PREC_FP64
        return {"dense_apply": measure_dense_only(rr, dev, stream,
                                                  dict(stream=stream, precision=prec))}
    X, y, _, p = synth.workload(args.workload)
    N, F, nnz, k, lams = X.n_rows, X.n_cols, X.nnz, p["k"], p["lambdas"]
    row_ptr = torch.as_tensor(X.row_ptr, device=dev)
    col_idx = torch.as_tensor(X.col_idx, device=dev)
    y_dev = torch.as_tensor(y, device=dev)
    W = [torch.empty(F, dtype=torch.float64, device=dev) for _ in lams]

    prec = rr.RR_PREC_MIXED if args.precision == "mixed" else rr.RR_PREC_FP64
    opts = dict(seed=p["seed"], stream=stream, precision=prec, max_restarts=20,
                split_head=args.split_head,
                use_graphs=0 if args.no_graphs else 1,
                gather={"auto": rr.RR_GATHER_AUTO, "lanes": rr.RR_GATHER_LANES,
                        "staged": rr.RR_GATHER_STAGED,
                        "lanes-staged": rr.RR_GATHER_LANES_STAGED}[args.gather])

    if args.profile_apply:
        h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], k, **opts)
        v = torch.randn(F, dtype=torch.float64, device=dev)
        z = torch.empty(F, dtype=torch.float64, device=dev)
        for _ in range(3):
            rr.rr_apply(h, v, z)
        torch.cuda.synchronize(dev)
        torch.cuda.cudart().cudaProfilerStart()
        for _ in range(args.profile_apply):
            rr.rr_apply(h, v, z)
        torch.cuda.synchronize(dev)
        torch.cuda.cudart().cudaProfilerStop()
        rr.rr_free(h)
        return {"profile_apply": args.profile_apply, "workload": args.workload}
    if args.roofline_only:
        return {"workload": args.workload, "precision": args.precision,
                "roofline": measure_roofline(rr, row_ptr, col_idx, N, F, nnz, k, lams, opts, dev,
                                             stream, args.workload)}
    if args.only_eigen:
        return {"coarse_eigen": measure_eigen(rr, row_ptr, col_idx, N, F, k, lams, opts, dev,
                                              stream, y_dev)}
    if args.only_leader:
        tol2s = [float(t) for t in args.leader_tol2.split(",") if t] or LEADER_TOL2
        return {"leader": measure_leader(rr, row_ptr, col_idx, N, F, lams, opts, dev, y_dev,
                                         tol2s, kmeans_same_k=True)}
    if args.only_bayes:
        return {"bayes": measure_bayes(rr, row_ptr, col_idx, N, F, k, lams[0], opts, dev, y_dev)}
    if args.only == "batched":
        b = measure_batched(rr, X, row_ptr, col_idx, k, opts, dev, stream, world,
                            args.batch_targets)
        b.pop("_samples", None)
        return {"batched": b}
    if args.only == "many":
        return {"many": measure_many(rr, dev, stream, opts, args.many_workload)}
    if args.only == "learned":
        return {"learned": measure_learned(rr, X, row_ptr, col_idx, k, opts, dev, stream,
                                           n_pairs=args.pairs)}

    def step(host=None):
        if host is None:
            h = rr.rr_setup(row_ptr, col_idx, N, F, lams[0], k, **opts)
            yd = y_dev
        else:
            h = rr.rr_setup(host["rp"], host["ci"], N, F, lams[0], k, **opts)
            yd = host["y"].to(dev, non_blocking=True)
        if args.no_graphs:
            # host-issued loops (the profiling form): one weight after the other,
            # the coarse levels of the others built while the first one solves
            rr.rr_prepare_lambdas(h, lams[1:])
            infos = []
            for j, lam in enumerate(lams):
                if j:
                    rr.rr_set_lambda(h, lam)
                infos.append(rr.rr_solve(h, yd, W[j], tol=TOL))
        else:
            # a fork per further weight (its coarse factor starts at once on its
            # own stream), then the weights' CG loops as branches of one graph
            forks = [rr.rr_fork_lambda(h, lam) for lam in lams[1:]]
            res = rr.rr_solve_many([h] + forks, [yd] * len(lams), W, tol=TOL, stream=stream)
            infos = res["infos"]
            for inf in infos:
                inf["status"] = res["status"]   # the call's status (RR_OK: every weight converged)
            for f in forks:
                rr.rr_free(f)
        if host is not None:
            for j in range(len(lams)):
                host["w"][j].copy_(W[j], non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()
        rr.rr_free(h)
        return infos

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    if args.profile_step:
        l0 = rr.rr_launch_count()
        infos = step()
        torch.cuda.synchronize(dev)
        return {"profile_step": args.workload, "gpu_launches": rr.rr_launch_count() - l0,
                "iters": [i["iters"] for i in infos]}
    parity_proc = None
    tmpdir = tempfile.mkdtemp(prefix="rr_parity_")
    if rank == 0 and args.workload == WORKLOAD and not args.no_parity:
        parity_proc, parity_path = start_parity(X, y, p, tmpdir, batch=not args.no_batch)
    for _ in range(max(3, args.warmup)):
        infos = step()
    for inf in infos:
        assert inf["status"] == "RR_OK" and inf["true_rel_res"] <= TOL, inf

    # ---- timed region: device-resident inputs
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    l0 = rr.rr_launch_count()
    all_infos = []
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for s in range(args.steps):
            all_infos.append(step())
            ev[s + 1].record(stream)
        torch.cuda.synchronize(dev)
    launches = rr.rr_launch_count() - l0
    barrier()
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = sum(step_ms)
    total_ms = slowest_over_ranks(total_ms, world, dev)
    value = total_ms / 1000.0 / args.steps

    roofline = measure_roofline(rr, row_ptr, col_idx, N, F, nnz, k, lams, opts, dev, stream,
                                args.workload)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host = {"rp": torch.as_tensor(X.row_ptr).pin_memory().numpy(),
                "ci": torch.as_tensor(X.col_idx).pin_memory().numpy(),
                "y": torch.as_tensor(y).pin_memory(),
                "w": [torch.empty(F, dtype=torch.float64).pin_memory() for _ in lams]}
        step(host)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(host)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        e_ms = slowest_over_ranks(t0.elapsed_time(t1) / args.steps, world, dev)
        e2e = {"value": round(e_ms / 1000.0, 5), "unit": "s",
               "h2d_bytes_per_step": 8 * (N + 1) + 4 * nnz + 8 * N,
               "d2h_bytes_per_step": 8 * F * len(lams)}

    batched = many = learned = tlfcg = eig = bayes = leader = None
    if not args.no_eigen and args.workload == WORKLOAD:
        eig = measure_eigen(rr, row_ptr, col_idx, N, F, k, lams, opts, dev, stream, y_dev)
    if not args.no_bayes and args.workload == WORKLOAD:
        bayes = measure_bayes(rr, row_ptr, col_idx, N, F, k, lams[0], opts, dev, y_dev)
    if not args.no_leader and args.workload == WORKLOAD:
        leader = measure_leader(rr, row_ptr, col_idx, N, F, lams, opts, dev, y_dev, LEADER_TOL2)
    if not args.no_tlfcg:
        tlfcg = measure_tlfcg(rr, row_ptr, col_idx, N, F, k, lams, opts, y_dev)
    if not args.no_batch and args.workload == WORKLOAD:
        batched = measure_batched(rr, X, row_ptr, col_idx, k, opts, dev, stream, world,
                                  args.batch_targets)
    if not args.no_many:
        many = measure_many(rr, dev, stream, opts)
    if not args.no_learned and args.workload == WORKLOAD:
        learned = measure_learned(rr, X, row_ptr, col_idx, k, opts, dev, stream, n_pairs=args.pairs)

    small = measure_small_fp64(rr, dev) if not args.no_small else None
    parity = None
    if parity_proc is not None:
        samples = batched.pop("_samples", None) if batched else None
        parity, bpar = finish_parity(parity_proc, parity_path, [w.cpu().numpy() for w in W], lams,
                                     W_batch=samples)
        if batched is not None:
            batched["parity"] = bpar
    elif batched is not None:
        batched.pop("_samples", None)
    last = all_infos[-1]
    out = {
        "metric": METRIC, "value": round(value, 5), "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded Zipf s=1.1 binary CSR, y = X w* + N(0, 0.1^2))",
        "config": {"workload": args.workload, "n_rows": N, "n_cols": F, "nnz": nnz, "k": k,
                   "lambdas": list(lams), "tol": TOL, "precision": args.precision,
                   "method": "two-level PCG: k-means++ clusters, SA prolongation, Cholesky "
                             "coarse solve, symmetric damped-Jacobi V(1,1)",
                   "l2": "inputs larger than L2 (CSR+CSC indices 8*nnz bytes)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "breakdown": {"setup_ms": round(last[0]["setup_ms"], 2),
                      "setup_phase_ms": dict(zip(
                          ["copy_validate", "csc_build", "kmeanspp_seed", "lloyd", "clusters",
                           "coarse_gram", "coarse_factor", "sliced_patterns"],
                          [round(v, 2) for v in last[0]["setup_phase_ms"]])),
                      "solve_ms": ([round(i["solve_ms"], 2) for i in last] if args.no_graphs
                                   else round(last[0]["solve_ms"], 2)),
                      "solve_form": ("one weight after the other (rr_set_lambda)" if args.no_graphs
                                     else "concurrent: rr_fork_lambda per further weight, "
                                          "rr_solve_many over the three"),
                      "iters": [i["iters"] for i in last],
                      "restarts": [i["restarts"] for i in last],
                      "true_rel_res": [i["true_rel_res"] for i in last],
                      "kmeans_iters": last[0]["kmeans_iters"], "k_eff": last[0]["k_eff"],
                      "gram_tensor_cores": bool(last[0]["gram_tensor_cores"]),
                      "gather_kernel": {"X": "staged" if last[0]["gather_staged"] & 1 else "lanes",
                                        "Xt": "staged" if last[0]["gather_staged"] & 2 else "lanes"},
                      "step_ms": [round(t, 3) for t in step_ms]},
        "e2e": e2e, "roofline": roofline, "clocks": clk.summary(), "gpu_launches": launches,
        "batched": batched, "many": many, "learned": learned, "tlfcg": tlfcg,
        "parity": parity, "small_fp64": small, "coarse_eigen": eig, "bayes": bayes,
        "leader": leader,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's own counts where recorded (its FP64 PCG needs fewer
        # iterations than the mixed-precision GPU solves), else the GPU's
        iters, km_iters = REF_COUNTS.get(args.workload, ([i["iters"] for i in last],
                                                         last[0]["kmeans_iters"]))
        out["cpu_baseline"] = cpu_baseline(X, y, p, iters, km_iters, last[0]["k_eff"])
        allc = cpu_baseline(X, y, p, iters, km_iters, last[0]["k_eff"], cores=os.cpu_count() or 1)
        out["cpu_baseline"]["all_cores"] = {key: allc.get(key) for key in
                                            ("value", "cores", "sample_wall_s", "parts_s")}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


# ---------------------------------------------------------------- the oracle on host cores

SAMPLE_NOTE = ("component sample of the FP64 oracle at full size, extrapolated to one step: CSC "
               "build (full), k-means++ seeding (first 8 centres, x k/8), one Lloyd assignment "
               "step (full, x the Lloyd steps taken), coarse counts (full) and 8 columns of the "
               "Gram (x k_eff/8), one Cholesky (x lambdas), two two-level PCG iterations (x the "
               "iterations taken)")


def _oracle_sample(npz_path, k, lam, iters, kmeans_iters, k_eff, seed):
    """Runs in a child process with one BLAS thread; returns the extrapolated seconds."""
    import numpy as np
    from oracle import kmeans as km
    from oracle import krylov, twolevel
    from oracle import sparse as osp

    d = np.load(npz_path)
    rp, ci, y = d["row_ptr"], d["col_idx"], d["y"]
    N, F = len(rp) - 1, int(d["n_cols"])
    T = {}
    t = time.perf_counter()
    cp, ri = osp.csc_pattern(N, F, rp, ci)
    T["csc"] = time.perf_counter() - t
    t = time.perf_counter()
    seeds = km.kmeanspp_binary(N, F, rp, ci, cp, ri, 8, seed)
    T["seed_per_centre"] = (time.perf_counter() - t) / 8
    t = time.perf_counter()
    labels, _ = km.lloyd_binary(N, F, rp, ci, cp, ri, seeds, 1)
    T["lloyd_step"] = time.perf_counter() - t
    # a clustering with k_eff clusters for the coarse-level timings (cost depends on sizes only)
    lab = (np.arange(F) % k_eff).astype(np.int32)
    t = time.perf_counter()
    C = twolevel.coarse_counts(N, F, rp, ci, lab, k_eff)
    Ct = C.T.tocsr()
    T["counts"] = time.perf_counter() - t
    t = time.perf_counter()
    cols = C[:, :8].toarray()
    _ = Ct @ cols
    T["gram_per_col"] = (time.perf_counter() - t) / 8
    rng = np.random.default_rng(0)
    B = rng.standard_normal((k_eff, k_eff))
    Ac = B @ B.T / k_eff + np.eye(k_eff)
    t = time.perf_counter()
    L = twolevel.cholesky(Ac)
    T["cholesky"] = time.perf_counter() - t
    M = osp.from_csr(N, F, rp, ci)
    n_S = np.bincount(lab, minlength=k_eff).astype(np.int64)
    s = twolevel.prolong_scale(n_S)
    dd = osp.col_sq_norms(M) + lam
    two = twolevel.TwoLevel(M, lam, lab, n_S, s, None, Ac, L, dd, 1.0 / 200.0,
                            seeds, 1)
    b = osp.rhs(M, y)
    t = time.perf_counter()
    krylov.pcg(two.A, two.apply, b, tol=1e-30, max_iter=2, max_restarts=0)
    T["pcg_iter"] = (time.perf_counter() - t) / 2.0   # includes the final true-residual check
    total = (T["csc"] + k * T["seed_per_centre"] + kmeans_iters * T["lloyd_step"] + T["counts"]
             + k_eff * T["gram_per_col"] + len(iters) * T["cholesky"] + sum(iters) * T["pcg_iter"])
    return total, T


def cpu_baseline(X, y, p, iters, kmeans_iters, k_eff, quiet=False, cores=1):
    """Times the oracle sample in a child process with `cores` threads (the
    oracle's only threaded part is the Lloyd assignment step; numpy's BLAS
    gets the same count)."""
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "x.npz")
        np.savez(path, row_ptr=X.row_ptr, col_idx=X.col_idx, y=y, n_cols=X.n_cols)
        env = dict(os.environ, OMP_NUM_THREADS=str(cores), OPENBLAS_NUM_THREADS=str(cores),
                   MKL_NUM_THREADS=str(cores), CUDA_VISIBLE_DEVICES="")
        code = ("import json,sys; sys.path.insert(0, %r); import bench; "
                "tot, T = bench._oracle_sample(%r, %d, %r, %r, %d, %d, %d); "
                "print(json.dumps({'total': tot, 'parts': T}))" %
                (ROOT, path, p["k"], float(p["lambdas"][0]), list(iters), kmeans_iters, k_eff,
                 p["seed"]))
        t0 = time.perf_counter()
        res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             cwd=ROOT)
        wall = time.perf_counter() - t0
    if res.returncode != 0:
        return {"value": None, "unit": "s", "cores": cores, "kind": "oracle",
                "error": res.stderr.strip().splitlines()[-1:] if res.stderr else "failed"}
    r = json.loads(res.stdout.strip().splitlines()[-1])
    return {"value": round(r["total"], 3), "unit": "s", "cores": cores, "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": SAMPLE_NOTE, "sample_wall_s": round(wall, 1),
            "parts_s": {k2: round(v, 4) for k2, v in r["parts"].items()}}


# Lloyd steps and FP64 two-level PCG iterations per lambda of the oracle's own
# full solve of the bench workload (a ten-minute run: 16 Lloyd steps, k_eff =
# 1000, 65 / 65 / 50 iterations, no refinement restart); the oracle counts them
# itself on workloads small enough to solve within the arm's run.
REF_COUNTS = {"zipf_200000x100000": ([65, 65, 50], 16)}


def oracle_counts(X, y, p):
    """PCG iterations per lambda and Lloyd steps of the oracle's full solve."""
    from oracle import krylov, twolevel
    from oracle import sparse as osp
    two = twolevel.setup_binary(X.n_rows, X.n_cols, X.row_ptr, X.col_idx, p["lambdas"][0], p["k"],
                                seed=p["seed"])
    b = osp.rhs(two.M, y)
    iters = []
    for lam in p["lambdas"]:
        t = two if lam == two.lam else two.with_lambda(lam)
        iters.append(krylov.pcg(t.A, t.apply, b, tol=TOL).iters)
    return iters, two.kmeans_iters


def run_reference(args, rank, world):
    """The oracle arm: each timed step re-measures the bounded sample."""
    if rank != 0:
        return None
    from gen import synth
    X, y, _, p = synth.workload(args.workload)
    if "RR_REF_ITERS" in os.environ:
        iters = [int(v) for v in os.environ["RR_REF_ITERS"].split(",")]
        km_iters = int(os.environ.get("RR_REF_KMEANS_ITERS", "16"))
        source = "RR_REF_ITERS"
    elif args.workload in REF_COUNTS:
        iters, km_iters = REF_COUNTS[args.workload]
        source = "recorded oracle solve"
    else:
        iters, km_iters = oracle_counts(X, y, p)
        source = "oracle solve"
    vals, last = [], None
    for _ in range(args.steps):
        last = cpu_baseline(X, y, p, iters, km_iters, p["k"])
        vals.append(last["value"])
    v = statistics.mean(vals)
    return {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(v * 1000, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "k": p["k"], "lambdas": list(p["lambdas"]),
                       "tol": TOL, "iters_assumed": iters, "kmeans_iters_assumed": km_iters,
                       "counts_from": source},
            "cpu_baseline": dict(last, value=round(v, 3)),
            "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
