#!/usr/bin/env python3
"""Benchmark of the l1-LS hot path on one GB300 (or N replicas under torchrun).

Workload: the large single instance (m = 2^25, n = 2^24, about 8 nonzeros per column, FP32
values, int32 indices, kappa(A) = 1e4, x* 1% nonzeros, tau = 1).  One step is one fused FISTA
iteration: K1 (A x with the momentum / residual epilogue and FP64 gap partials) and K2 (A^T r
with the shrinkage / momentum epilogue and the FP64 certificate), i.e. both products.

value   = algorithmic bytes of the two products with their fused vector traffic per
          iteration / device time per iteration (CUDA events on the launching stream),
          summed over ranks (weak scaling: one instance per GPU).
e2e     = the same quantity through l1ls_solve_fista with HOST buffers: every step is a
          warm-started 32-iteration solve from a pinned host x0 to a pinned host x_out.
roofline: the dominant kernel (K1 or K2) against the measured HBM copy bandwidth.
cpu_baseline / --impl reference: the FP64 oracle (numpy + scipy) on a sample of the same
          recipe, timed on the host cores, in the same unit.
"""

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the serving leg runs up to 16 slots on their own streams: 32 hardware work queues instead of
# the default 8 keep the streams from sharing queues (read when CUDA initialises)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "Ax/ATy HBM GB/s (fused FISTA iteration)"
UNIT = "GB/s"
FALLBACK_HBM = 6800.0
E2E_ITERS = 32
KERNEL_SOURCES = ["spmv.cuh", "fista.cu", "common.cuh"]


def bytes_per_iteration(m, n, nnz, value_bytes=4, vec_bytes=4, paired=True):
    """Algorithmic bytes of K1 and K2 (FP32 values and products, FP64 iterates).

    Stored matrix: with one left rotation the rows 2p and 2p+1 share their columns, so each
    orientation stores one int32 index per pair of entries and the two values:
    nnz/2 * (4 + 2 v) bytes plus the pointers (m/2 + 1 for rows, n + 1 for columns).
    K1: matrix (row pairs) + x gathered once (n FP32) + A x_{k-2} read, b read, A x_{k-1}
        written, r written (4 m-vectors).
    K2: matrix (columns) + r gathered once (m FP32) + x_{k-1}, x_{k-2} read and x_k written
        (8 bytes each: float-float pairs, the hi half being what K1 gathers).
    """
    if paired:
        mat = (nnz // 2) * (4 + 2 * value_bytes)
        p1, p2 = (m // 2 + 1) * 4, (n + 1) * 4
    else:
        mat = nnz * (4 + value_bytes)
        p1, p2 = (m + 1) * 4, (n + 1) * 4
    k1 = mat + p1 + n * vec_bytes + 4 * m * vec_bytes
    k2 = mat + p2 + m * vec_bytes + 3 * n * 8
    return k1, k2


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1503_03520_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it still matches."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("bytes_per_launch", {}).get(kernel)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


CPU_SAMPLE_LOG2N = 20     # the oracle's sample of the C2 recipe: n = 2^20, m = 2^21

_ORACLE_TIMING = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
import workloads as W
from oracle.generator import GenParams, generate
from oracle import solvers
p = W.c2_scaled(%(log2n)d, seed=%(seed)d)
t0 = time.time()
inst = generate(GenParams.from_dict(p))
tgen = time.time() - t0
A, b = inst.A, inst.b
solvers.fista(A, b, 1.0, inst.lipschitz, 0.0, %(warmup)d)
steps = %(steps)d
if steps <= 0:
    t = time.time(); solvers.fista(A, b, 1.0, inst.lipschitz, 0.0, 2); one = (time.time() - t) / 2
    steps = max(3, int(%(budget)f / max(one, 1e-6)))
go = %(go)r
if go:
    open(os.path.join(go, "ready.%%d" %% os.getpid()), "w").close()
    while not os.path.exists(os.path.join(go, "go")):
        time.sleep(0.01)
t = time.time()
r = solvers.fista(A, b, 1.0, inst.lipschitz, 0.0, steps)
t1 = time.time()
print(json.dumps(dict(m=A.shape[0], n=A.shape[1], nnz=int(A.nnz), steps=steps, seconds=t1 - t, start=t, end=t1,
                      gen_seconds=tgen)))
"""


def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    return env


def cpu_oracle_iterations(log2n, warmup, steps, budget_s):
    """Time oracle FISTA iterations in a fresh single-threaded Python process."""
    code = _ORACLE_TIMING % dict(root=ROOT, log2n=log2n, seed=0, warmup=max(warmup, 1), steps=steps,
                                 budget=budget_s, go="")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=_oracle_env(), timeout=900)
    if out.returncode != 0:
        raise RuntimeError("oracle timing failed: " + out.stderr[-2000:])
    d = json.loads(out.stdout.strip().splitlines()[-1])
    k1, k2 = bytes_per_iteration(d["m"], d["n"], d["nnz"])
    per_iter = d["seconds"] / d["steps"]
    d["value"] = (k1 + k2) / per_iter / 1e9
    d["ms_per_step"] = per_iter * 1e3
    d["cores"] = 1
    return d


def host_cores_for_oracle(bytes_per_process=1.6e9):
    """Host cores the all-cores oracle uses: every core, bounded by the available memory (one
    single-threaded oracle process per core, each holding its own instance)."""
    cores = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(l.split()[1]) * 1024 for l in f if l.startswith("MemAvailable"))
        cores = max(1, min(cores, int(0.6 * avail / bytes_per_process)))
    except Exception:
        pass
    return cores


def cpu_oracle_all_cores(log2n, warmup, steps, budget_s, cores=None):
    """The oracle as it stands on all host cores: one single-threaded oracle process per core,
    each on its own seeded instance of the sample (independent replicas, as the GPU ranks are),
    released together once every process has generated its instance and warmed up.  value =
    the algorithmic bytes of all processes' iterations / (last end - first start)."""
    import tempfile
    cores = cores or host_cores_for_oracle()
    with tempfile.TemporaryDirectory() as go:
        procs = []
        for c in range(cores):
            code = _ORACLE_TIMING % dict(root=ROOT, log2n=log2n, seed=c, warmup=max(warmup, 1), steps=steps,
                                         budget=budget_s, go=go)
            procs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                          stderr=subprocess.PIPE, text=True, env=_oracle_env()))
        t0 = time.time()
        while sum(f.startswith("ready.") for f in os.listdir(go)) < cores:
            if any(p.poll() not in (None, 0) for p in procs) or time.time() - t0 > 900:
                for p in procs:
                    p.kill()
                raise RuntimeError("all-cores oracle timing failed before the start")
            time.sleep(0.05)
        open(os.path.join(go, "go"), "w").close()
        rows = []
        for p in procs:
            out, err = p.communicate(timeout=900)
            if p.returncode != 0:
                raise RuntimeError("all-cores oracle timing failed: " + err[-2000:])
            rows.append(json.loads(out.strip().splitlines()[-1]))
    k1, k2 = bytes_per_iteration(rows[0]["m"], rows[0]["n"], rows[0]["nnz"])
    span = max(r["end"] for r in rows) - min(r["start"] for r in rows)
    total_steps = sum(r["steps"] for r in rows)
    return {"value": (k1 + k2) * total_steps / span / 1e9, "cores": cores, "steps": total_steps,
            "seconds": span, "ms_per_step": span / max(r["steps"] for r in rows) * 1e3, "m": rows[0]["m"],
            "n": rows[0]["n"], "nnz": rows[0]["nnz"]}


def cpu_baseline_line(single, multi, log2n):
    what = ("oracle FISTA iterations (numpy + scipy.sparse, FP64) on the n=2^%d, m=2^%d instance of the same "
            "recipe" % (log2n, log2n + 1))
    return {"value": multi["value"], "unit": UNIT, "cores": multi["cores"], "kind": "oracle",
            "sample": "%s: %d single-threaded processes, one per host core, each on its own seeded instance, "
                      "%d iterations in %.1f s together" % (what, multi["cores"], multi["steps"], multi["seconds"]),
            "single_thread": {"value": single["value"], "unit": UNIT, "cores": 1,
                              "sample": "%s: %d iterations in %.1f s, one thread" % (what, single["steps"],
                                                                                      single["seconds"])}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    log2n = CPU_SAMPLE_LOG2N
    steps = args.steps
    single = cpu_oracle_iterations(log2n, args.warmup, steps, 0.0)
    multi = cpu_oracle_all_cores(log2n, args.warmup, steps, 0.0)
    line = {"metric": METRIC, "value": multi["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": args.warmup, "ms_per_step": multi["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (generator of Sec. 3-6)",
            "impl": "reference",
            "config": {"workload": "c2: m=2^25, n=2^24, ~8 nnz/col, FP32 values, kappa(A)=1e4, x* 1%, tau=1",
                       "sample": "n=2^%d, one oracle FISTA iteration per step and process" % log2n,
                       "l2": "inputs larger than L2"},
            "cpu_baseline": cpu_baseline_line(single, multi, log2n),
            "e2e": {"value": multi["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(value, dist, device="cuda"):
    """The largest value over all ranks (the job's time is its slowest rank's); value itself
    without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def pcg_bytes_per_iteration(m, n, nnz):
    """Algorithmic bytes of one pdNCG PCG iteration with FP32 values in paired storage: C1 (the
    row pairs, z gathered, A p read and written), C2 (the columns, A p gathered as one float2 per
    row pair, z, p and the curvature read, p and Hp written), C3 (d, p, Hp, M^-1 read and the
    float-float residual read; d, z written and the residual written)."""
    mat = (nnz // 2) * 12
    c1 = mat + (m // 2 + 1) * 4 + 4 * n + 8 * m
    c2 = mat + (n + 1) * 4 + 4 * m + 12 * n + 8 * n
    c3 = 16 * n + 8 * n + 8 * n + 8 * n
    return c1 + c2 + c3


def mf_pcg_bytes_per_iteration(n):
    """Algorithmic bytes of one PCG iteration of pdNCG on a matrix-free instance (FP32 vectors):
    the product sweep (z, p_old, the curvature and sigma read, p and Hp written: 24n; A^T A p
    = R Sigma^2 R^T p needs no m-vector) and the update (p, Hp, M^-1 read, d read and written,
    the float-float residual read and written, z written: 40n)."""
    return 24 * n + 40 * n


def pcg_iteration_timing(inst, m, n, nnz, lo=16, hi=144, bytes_fn=None):
    """Time per PCG iteration of pdNCG: one Newton step from a point near x* with the relative
    residual target 1e-30 (PCG runs to its cap) at two caps; the difference of the two solve
    times over the difference of the iteration counts (whole CUDA-graph chunks of 16, so the
    host checks cancel)."""
    import numpy as np
    import torch
    xs = inst.xstar()
    rng = np.random.default_rng(0)
    # x0 and x_out on the device: host copies of n doubles would add noise to both times
    x0 = torch.tensor(xs * (1.0 + 0.01 * rng.standard_normal(xs.size)) + 1e-3 * rng.standard_normal(xs.size),
                      device="cuda")
    xo = torch.empty_like(x0)
    out = {}
    for k in (lo, hi):
        best = None
        for _ in range(3):
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, r = inst.solve_pdncg(x0=x0, x_out=xo, tau=1.0, tol=0.0, max_iter=1, pcg_max=k, pcg_rtol=1e-30,
                                    mu_start=1e-5, check_every=16, allow=(4, 5))
            el = time.perf_counter() - t
            best = el if best is None else min(best, el)
        out[k] = (best, r["cg_iters"])
    iters = out[hi][1] - out[lo][1]
    if iters <= 0:
        return None
    ms = (out[hi][0] - out[lo][0]) / iters * 1e3
    b = bytes_fn(n) if bytes_fn else pcg_bytes_per_iteration(m, n, nnz)
    peak, src = measured_hbm_peak()
    return {"ms": ms, "algorithmic_bytes": b, "gbs": b / (ms * 1e-3) / 1e9, "frac": b / (ms * 1e-3) / 1e9 / peak,
            "peak_source": src, "method": "(t(%d) - t(%d)) / %d PCG iterations of one Newton step" % (hi, lo, iters)}


def rank_workload(log2n, rank):
    """The instance each rank times: the same recipe, its own seed (replicas, no collective)."""
    import workloads as W
    return W.c2_scaled(log2n, seed=rank)


def batch_bytes_per_step(m, n, nnz):
    """Algorithmic bytes of one step of the batched kernel for one instance (FP32 values in
    paired storage, float-float vectors as interleaved {hi, lo} pairs).  Row phase: row-pair
    pointers, indices and values, the iterate gathered as one pair per column (8n), A x_{k-1}
    read and A x_k written as pairs (16m), b (4m), the residual's {hi, lo} written (8m).
    Column phase: column pointers, indices and values, the residual gathered (8m), both iterates
    read and the new one written (24n)."""
    mat = 4 * (nnz // 2) + 4 * nnz
    rows = mat + 4 * (m // 2 + 1) + 8 * n + 16 * m + 4 * m + 8 * m
    cols = mat + 4 * (n + 1) + 8 * m + 24 * n
    return rows + cols


def batch_form(l1, W, ctx, iters_per_tau):
    """C4: 256 instances along 16-tau paths in the batched kernel, against the same paths
    solved one instance at a time with FP64 values (a 1-in-16 subsample), equal tolerance and
    iteration caps."""
    import numpy as np
    import torch
    params = W.c4_batch(256)
    insts = [ctx.generate(p) for p in params]
    taus = np.array([W.c4_tau_path(i.info["lam_max"]) for i in insts])
    b = l1.Batch(ctx, insts)
    opts = dict(tol=1e-6, max_iter=iters_per_tau, restart=1)
    t = time.perf_counter()
    res = b.solve_path(taus, **opts)
    el = time.perf_counter() - t
    st = b.stats()
    sched = b.schedule()
    # the kernel's bandwidth: algorithmic bytes of every instance-iteration run over the device
    # time of all steps; once for the whole path, once for 64 iterations at the last (smallest)
    # tau, where no instance certifies so early (the schedule is already chosen: no probes)
    ib = [batch_bytes_per_step(i.m, i.n, i.nnz) for i in insts]
    path_bytes = sum(ib[k] * r["iters"] for k, rr in enumerate(res) for r in rr)
    res_all = b.solve_path(taus[:, -1:], tol=1e-300, max_iter=64, restart=1, allow=(4, 5))
    st_all = b.stats()
    all_bytes = sum(ib[k] * rr[0]["iters"] for k, rr in enumerate(res_all))
    all_iters = sum(rr[0]["iters"] for rr in res_all)
    peak, src = measured_hbm_peak()
    b.free()
    it = sum(r["iters"] for rr in res for r in rr)
    ok = sum(r["status"] == 0 for rr in res for r in rr)
    ok_by_tau = [sum(rr[j]["status"] == 0 for rr in res) for j in range(taus.shape[1])]
    for i in insts:
        i.free()
    sub = list(range(0, 256, 16))
    t_one, it_one, ok_one = 0.0, 0, 0
    for i in sub:
        inst = ctx.generate(dict(params[i], value_dtype="f64"))
        x0 = None
        torch.cuda.synchronize()
        t = time.perf_counter()
        for tau in taus[i]:
            x0, r = inst.solve_fista(tau=float(tau), x0=x0, allow=(4, 5), **opts)
            it_one += r["iters"]
            ok_one += r["status"] == 0
        t_one += time.perf_counter() - t
        inst.free()
    rate, rate_one = it / el, it_one / t_one
    cert_rate, cert_rate_one = ok / el, ok_one / t_one
    return {"workload": "c4: 256 instances, n = 2^U[12,18], m = 2n, ~8/col, kappa 10^U[2,5], x* 1%%, 16 taus "
                        "0.9 lambda_max .. 1e-3, warm-started, tol 1e-6, at most %d FISTA iterations per tau"
                        % iters_per_tau,
            "batched": {"seconds": el, "instance_iterations": it, "instance_iterations_per_s": rate,
                        "certified": ok, "of": 256 * 16, "certified_per_s": cert_rate,
                        "certified_by_tau_index": ok_by_tau, "steps": st["steps"],
                        "ms_per_step": st["device_ms"] / max(1, st["steps"]), "schedule": sched,
                        "values": "FP32, float-float products and iterates"},
            "bandwidth": {"path": {"algorithmic_bytes": path_bytes, "device_ms": st["device_ms"],
                                   "gbs": path_bytes / (st["device_ms"] * 1e-3) / 1e9,
                                   "frac": path_bytes / (st["device_ms"] * 1e-3) / 1e9 / peak},
                          "last_tau_64_iterations": {"instance_iterations": all_iters, "steps": st_all["steps"],
                                                     "algorithmic_bytes": all_bytes, "device_ms": st_all["device_ms"],
                                                     "gbs": all_bytes / (st_all["device_ms"] * 1e-3) / 1e9,
                                                     "frac": all_bytes / (st_all["device_ms"] * 1e-3) / 1e9 / peak},
                          "peak_source": src,
                          "bytes": "batch_bytes_per_step of each instance times its iterations (includes the "
                                   "autotuner's probe steps in the path's device time)"},
            "one_at_a_time_fp64": {"seconds": t_one, "instances": len(sub), "instance_iterations": it_one,
                                   "instance_iterations_per_s": rate_one, "certified": ok_one,
                                   "of": len(sub) * 16, "certified_per_s": cert_rate_one,
                                   "api": "l1ls_solve_fista per instance and tau"},
            "speedup_instance_iterations": rate / rate_one,
            "speedup_certified_per_s": cert_rate / max(cert_rate_one, 1e-12)}


SERVE_RATES = (10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0)


def serve_form(l1, W, count, rates, log2n_hi, slots=16):
    """C5: Poisson arrivals into the serving loop (`slots` slots, FP32 values, float-float FISTA
    products) against the same requests served FIFO one at a time with FP64 values (one slot),
    at each arrival rate.  The request sequence is the same at every rate (arrival times of the
    unit-rate sequence divided by the rate).  Both arms stop a request at the same iteration
    caps (no time limits), so a request is certified in both or fails in both up to the
    rounding of its certificate; certified solves per second count requests certified to the
    1e-6 gap over the span from the first arrival to the last completion; latency is from
    arrival to completion."""
    import numpy as np
    reqs = W.c5_requests(count, 1.0, log2n_hi=log2n_hi)

    def run(dtype, slots, accum, rate, mf_pdncg=False):
        ctx = l1.Context(0)
        ctx.serve_config(slots=slots)
        # iteration caps, not time limits: the same requests finish (or stop) in both runs
        of = dict(tol=1e-6, max_iter=5000, restart=1, accum=accum)
        op = dict(tol=1e-6, max_iter=30, pcg_max=300, accum=accum)
        t0 = time.perf_counter()
        tickets = []
        for r in reqs:
            due = r["t"] / rate
            now = time.perf_counter() - t0
            if due > now:
                time.sleep(due - now)
            o = of if r["method"] == "fista" else op
            p = dict(r["params"], value_dtype=dtype)
            if mf_pdncg and r["method"] == "pdncg" and p["m"] >= p["n"]:
                p["matrix_free"] = 1    # A by its factors (FP64 gradient, FP32 PCG product)
            tickets.append(ctx.submit(p, method=r["method"], tau=-r["tau_factor"], **o))
        out = []
        for t in tickets:
            while True:
                o = ctx.poll(t, wait_ms=100)
                if o is not None:
                    out.append(o)
                    break
        el = time.perf_counter() - t0 - reqs[0]["t"] / rate
        st = ctx.serve_stats()
        ctx.close()
        lat = np.array([o[1]["latency_s"] for o in out])
        ok = int(sum(o[0] == 0 for o in out))
        return {"seconds": el, "certified": ok, "of": len(out), "fraction_certified": ok / len(out),
                "certified_per_s": ok / el, "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "peak_running": st["peak_running"],
                "statuses": {l1.STATUS.get(k, str(k)): int(v) for k, v in
                             enumerate(np.bincount([o[0] for o in out], minlength=10)) if v}}

    table = []
    for rate in rates:
        served = run("f32", slots, 1, rate)
        served_mf = run("f32", slots, 1, rate, mf_pdncg=True)
        fifo = run("f64", 1, 0, rate)
        table.append({"rate_per_s": rate, "served": served, "served_matrix_free_pdncg": served_mf, "fifo_fp64": fifo,
                      "speedup_certified_per_s": served["certified_per_s"] / max(fifo["certified_per_s"], 1e-12),
                      "speedup_certified_per_s_matrix_free_pdncg":
                          served_mf["certified_per_s"] / max(fifo["certified_per_s"], 1e-12)})
    return {"workload": "c5: %d Poisson requests per rate, n = 2^U[10,%d], m in {n/2, 2n}, kappa 10^U[2,6], "
                        "x* 0.5-5%%, tau = 10^U[-2,0] lambda_max, FISTA (kappa <= 1e3, restart, at most 5000 "
                        "iterations) or pdNCG (at most 30 Newton steps of at most 300 PCG iterations), tol 1e-6"
                        % (count, log2n_hi),
            "slots": slots, "rates": table,
            "served_matrix_free_pdncg": "the served arm again, with the pdNCG requests of m >= n generated "
                                        "matrix-free (A by its factors: FP64 gradient, FP32 PCG product)",
            "best_speedup_certified_per_s": max(r["speedup_certified_per_s"] for r in table),
            "best_speedup_certified_per_s_matrix_free_pdncg":
                max(r["speedup_certified_per_s_matrix_free_pdncg"] for r in table)}


def mf_bytes_per_iteration(m, n, left=True):
    """Algorithmic bytes of one matrix-free FISTA iteration (FP32 vectors, float-float iterate):
    K1 = stage sweep (x hi, sigma, z: 12n) + rows of the left factor (perm 4m, z gathered 4n,
    A x read and written 8m, b 4m, the rotated residual scattered to P2^T order 4n);
    K2 = stage sweep of that n-vector with the FISTA epilogue (it and sigma 8n, both iterates
    read 16n, the new one written 8n)."""
    k1 = 12 * n + 8 * n + 16 * m
    k2 = 32 * n
    return k1, k2


def mf_form(l1, W, log2n, steps, warmup, solve_limit):
    """C2 with A in factored form (Algorithms MvPA / MvPAt on the device): FISTA iteration time,
    its HBM fraction, and the time to the 1e-6 gap, beside the stored-matrix path."""
    import torch
    ctx = l1.Context(0)
    params = dict(W.c2_scaled(log2n), matrix_free=1)
    inst = ctx.generate(params)
    m, n = inst.m, inst.n
    k1b, k2b = mf_bytes_per_iteration(m, n)
    stream = torch.cuda.current_stream()
    inst.fista_begin(tau=1.0, tol=0.0, max_iter=10 ** 12, stream=stream)
    inst.fista_step(warmup, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    kms = inst.fista_step(steps, timed=True, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    it_ms = e0.elapsed_time(e1) / steps
    inst.fista_end(stream=stream, allow=(4, 5))
    peak, _ = measured_hbm_peak()
    t = time.perf_counter()
    _, r = inst.solve_fista(tau=1.0, tol=W.C2_TOL, max_iter=200000, time_limit_s=solve_limit, stream=stream,
                            allow=(4, 5))
    el = time.perf_counter() - t
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, rp = inst.solve_pdncg(tau=1.0, tol=W.C2_TOL, max_iter=200, time_limit_s=solve_limit, stream=stream,
                             allow=(4, 5))
    elp = time.perf_counter() - t
    pcg = pcg_iteration_timing(inst, m, n, 0, bytes_fn=mf_pcg_bytes_per_iteration)
    out = {"workload": "c2 (m=2^%d, n=2^%d) with A not assembled: products by the stages of R, Sigma, "
                       "the permutation and the left rotations (FP32)" % (log2n + 1, log2n),
           "device_bytes": inst.info["device_bytes"], "iteration_ms": it_ms,
           "k1_ms": kms[0] / steps, "k2_ms": kms[1] / steps,
           "k1_bytes": k1b, "k2_bytes": k2b,
           "k1_frac": k1b / (kms[0] / steps * 1e-3) / 1e9 / peak, "k2_frac": k2b / (kms[1] / steps * 1e-3) / 1e9 / peak,
           "gbs": (k1b + k2b) / (it_ms * 1e-3) / 1e9,
           "fista_to_gap": {"tol": W.C2_TOL, "seconds": el, "iters": r["iters"], "rel_gap": r["rel_gap"],
                            "status": r["status_name"],
                            "rel_err_f": abs(r["f"] - inst.info["f_star"]) / inst.info["f_star"]},
           "pdncg_to_gap": {"tol": W.C2_TOL, "seconds": elp, "iters": rp["iters"], "cg_iters": rp["cg_iters"],
                            "rel_gap": rp["rel_gap"], "status": rp["status_name"],
                            "rel_err_f": abs(rp["f"] - inst.info["f_star"]) / inst.info["f_star"],
                            "pcg_iteration": pcg,
                            "method": "gradient and certificate by an FP64 sweep (A^T b - R Sigma^2 R^T x), "
                                      "PCG product by an FP32 sweep (A^T A = R Sigma^2 R^T)"}}
    inst.free()
    ctx.close()
    return out


def sec89_form(l1, W, log2n, newton_steps):
    """Sec. 8.9's huge-scale instance shape at n = 2^log2n on one GPU: pdNCG with the paper's
    mu = 1e-5 (no continuation below it) for a fixed number of Newton steps, reported as the
    relative error of x and f against the generator's x*, f* (the paper's measure there)."""
    import numpy as np
    ctx = l1.Context(0)
    rows = []
    for dt, mf in (("f64", 0), ("f32", 0), ("f32", 1)):
        inst = ctx.generate(dict(W.sec89(log2n, dt), matrix_free=mf))
        xs = inst.xstar()
        acc = 0 if dt == "f64" else 1
        tag = dt + (" matrix-free" if mf else "")
        for k in newton_steps:
            t = time.perf_counter()
            x, r = inst.solve_pdncg(tau=1.0, tol=0.0, max_iter=k, mu_min=1e-5, accum=acc, allow=(4, 5))
            rows.append({"values": tag, "newton": r["iters"], "pcg": r["cg_iters"], "seconds": time.perf_counter() - t,
                         "rel_err_x": float(np.linalg.norm(x - xs) / np.linalg.norm(xs)),
                         "rel_err_f": abs(r["f"] - inst.info["f_star"]) / inst.info["f_star"],
                         "rel_gap": r["rel_gap"]})
        for tol in (1e-4, 1e-6):   # to a certified gap with the defaults (continuation below mu allowed)
            t = time.perf_counter()
            x, r = inst.solve_pdncg(tau=1.0, tol=tol, max_iter=200, accum=acc, time_limit_s=30.0, allow=(4, 5))
            rows.append({"values": tag, "tol": tol, "status": r["status_name"], "newton": r["iters"],
                         "pcg": r["cg_iters"], "seconds": time.perf_counter() - t,
                         "rel_err_x": float(np.linalg.norm(x - xs) / np.linalg.norm(xs)),
                         "rel_err_f": abs(r["f"] - inst.info["f_star"]) / inst.info["f_star"],
                         "rel_gap": r["rel_gap"]})
        inst.free()
    ctx.close()
    return {"workload": "sec. 8.9 shape at n=2^%d (m=2n, sigma 0.1/100, theta 2pi/3, x* n/2^10 nonzeros -1e4/0.1), "
                        "pdNCG with mu = 1e-5" % log2n, "runs": rows}


def sec89_large_form(l1, W, log2n, newton_steps, tols=()):
    """Sec. 8.9's instance shape at the largest sizes one GPU holds, matrix-free (A = Sigma G^T
    is never assembled; O(n) memory): pdNCG for the paper's 8 Newton steps and more, with the
    paper's mu = 1e-5, the relative error of x against x* (Table 1's measure), device memory,
    time per PCG iteration and its HBM fraction."""
    import torch
    ctx = l1.Context(0)
    t = time.perf_counter()
    inst = ctx.generate(dict(W.sec89(log2n, "f32"), matrix_free=1))
    gen_s = time.perf_counter() - t
    xs = torch.tensor(inst.xstar(), device="cuda")
    x = torch.empty_like(xs)
    n = inst.n
    peak, src = measured_hbm_peak()
    rows = []
    for k in newton_steps:
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, r = inst.solve_pdncg(x_out=x, tau=1.0, tol=0.0, max_iter=k, mu_min=1e-5, allow=(4, 5))
        el = time.perf_counter() - t
        pcg_ms = 1e3 * el / max(1, r["cg_iters"])   # whole solve over its PCG iterations (an upper bound)
        rows.append({"newton": r["iters"], "pcg": r["cg_iters"], "seconds": el,
                     "rel_err_x": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs)),
                     "rel_err_f": abs(r["f"] - inst.info["f_star"]) / inst.info["f_star"], "rel_gap": r["rel_gap"],
                     "ms_per_pcg_iteration_upper": pcg_ms,
                     "pcg_frac_lower": mf_pcg_bytes_per_iteration(n) / (pcg_ms * 1e-3) / 1e9 / peak})
    for tol in tols:   # to a certified relative gap with the defaults (continuation below mu allowed)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, r = inst.solve_pdncg(x_out=x, tau=1.0, tol=tol, max_iter=200, allow=(4, 5))
        el = time.perf_counter() - t
        rows.append({"tol": tol, "status": r["status_name"], "newton": r["iters"], "pcg": r["cg_iters"],
                     "seconds": el, "rel_gap": r["rel_gap"],
                     "rel_err_x": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs)),
                     "rel_err_f": abs(r["f"] - inst.info["f_star"]) / inst.info["f_star"]})
    pcg = pcg_iteration_timing(inst, inst.m, n, 0, bytes_fn=mf_pcg_bytes_per_iteration)
    out = {"workload": "sec. 8.9 shape at n=2^%d (m=2^%d), matrix-free, FP32 PCG, FP64 gradient" % (log2n, log2n + 1),
           "generation_s": gen_s, "device_bytes": inst.info["device_bytes"], "pcg_iteration": pcg,
           "pdncg_work_bytes": 76 * n, "runs": rows, "peak_source": src,
           "x": "x0 = 0 and x_out on the device (the seconds include no host copy)",
           "paper": "Table 1: n = 2^30 on 64 processors, 1,923 s; 8 Newton steps, about 100 PCG iterations each, "
                    "relative error of order 1e-4"}
    inst.free()
    ctx.close()
    return out


def variants_form(l1, W, log2n, limit_s):
    """FISTA variants on the C2 recipe at n = 2^log2n (FP32 values, tau = 1, gap 1e-6): the
    paper's fixed L (= sigma_max^2 = 1, known exactly for these instances), the gradient
    restart, and backtracking on L from L0 = 1e-2 (factor 2; FP64 vectors, one host decision
    per trial)."""
    ctx = l1.Context(0)
    inst = ctx.generate(W.c2_scaled(log2n))
    f_star = inst.info["f_star"]
    rows = []
    for name, call in (("fixed_L", lambda: inst.solve_fista(tau=1.0, tol=W.C2_TOL, max_iter=10 ** 6,
                                                             time_limit_s=limit_s, allow=(4, 5))),
                       ("restart", lambda: inst.solve_fista(tau=1.0, tol=W.C2_TOL, max_iter=10 ** 6, restart=1,
                                                             time_limit_s=limit_s, allow=(4, 5))),
                       ("backtracking", lambda: inst.solve_fista_bt(1e-2, 2.0, tau=1.0, tol=W.C2_TOL,
                                                                     max_iter=10 ** 6, time_limit_s=limit_s,
                                                                     allow=(4, 5)))):
        t = time.perf_counter()
        _, r = call()
        el = time.perf_counter() - t
        row = {"variant": name, "status": r["status_name"], "iters": r["iters"], "products": r["products"],
               "seconds": el, "ms_per_iter": 1e3 * el / max(r["iters"], 1), "rel_gap": r["rel_gap"],
               "rel_err_f": abs(r["f"] - f_star) / f_star}
        if name == "backtracking":
            row.update({"L0": 1e-2, "eta": 2.0, "increases": r["ls_trials"], "L_final": r["L"]})
        rows.append(row)
    inst.free()
    ctx.close()
    return {"workload": "c2 recipe at m=2^%d, n=2^%d, tau=1, gap 1e-6, %g s limit" % (log2n + 1, log2n, limit_s),
            "runs": rows}


def osgen3_form(l1, W, log2n, limit_s):
    """Sec. 8.5's instances: x* by Procedure OsGen3 (gamma = 100, s1 = s2 = s/2, s = n/2^7),
    A = Sigma G^T (L = I, G = G2 G), n = 2^log2n, m = 2n, kappa(A^T A) = 1e2 .. 1e8, rotation
    angles 2 pi/10 and 2 pi/10^3: device generation time, kappa_rho(x*) at rho = 10 sigma_min^2
    (the paper's rho = 0.1 with its singular values shifted by 0.1), and FISTA to the 1e-6 gap
    (float-float products: with FP32 sums the certificate of these instances stalls near 1e-4
    while f is already within 1e-9 of f*)."""
    import math
    ctx = l1.Context(0)
    rows = []
    for theta in (2 * math.pi / 10, 2 * math.pi / 1e3):
        for kappa in (10.0, 1e2, 1e3, 1e4):
            n = 2 ** log2n
            params = W.params(m=2 * n, n=n, seed=5, kappa=kappa, right_stages=2, left_stages=0, theta=theta,
                              xstar_frac=2.0 ** -7, xstar_mode=2, gamma=100.0, value_dtype="f32")
            t = time.perf_counter()
            inst = ctx.generate(params)
            gen_s = time.perf_counter() - t
            krho = inst.kappa_rho(10.0 / kappa ** 2)
            t = time.perf_counter()
            _, r = inst.solve_fista(tau=1.0, tol=W.C2_TOL, max_iter=10 ** 6, accum=1, time_limit_s=limit_s,
                                    allow=(4, 5))
            el = time.perf_counter() - t
            rows.append({"theta": theta, "kappa_AtA": kappa ** 2, "s": inst.info["s"], "generate_s": gen_s,
                         "kappa_rho": krho, "fista_status": r["status_name"], "fista_iters": r["iters"],
                         "fista_s": el, "rel_gap": r["rel_gap"],
                         "rel_err_f": abs(r["f"] - inst.info["f_star"]) / inst.info["f_star"]})
            inst.free()
    ctx.close()
    return {"workload": "sec. 8.5 shape: OsGen3 x* (gamma 100, s = n/2^7), A = Sigma G^T, m=2^%d, n=2^%d, FP32 "
                        "values, FISTA (float-float products) %g s limit" % (log2n + 1, log2n, limit_s), "runs": rows}


def sweep_form(l1, W, stored_log2n, mf_log2n, steps, warmup):
    """C2's size sweep: the FISTA iteration on the C2 recipe at n = 2^k for the stored matrix
    (up to 2^27, the largest n whose nonzeros fit 32-bit offsets) and for the matrix-free
    products (up to 2^29): device time per iteration (CUDA events), algorithmic GB/s and the
    fraction of the measured HBM copy peak, and the instance's device memory."""
    import torch
    peak, _ = measured_hbm_peak()
    rows = []
    ctx = l1.Context(0)
    for mf, sizes in ((0, stored_log2n), (1, mf_log2n)):
        for k in sizes:
            inst = ctx.generate(dict(W.c2_scaled(k), matrix_free=mf))
            m, n, nnz = inst.m, inst.n, inst.nnz
            k1b, k2b = mf_bytes_per_iteration(m, n) if mf else bytes_per_iteration(m, n, nnz)
            stream = torch.cuda.current_stream()
            inst.fista_begin(tau=1.0, tol=0.0, max_iter=10 ** 12, stream=stream)
            inst.fista_step(warmup, stream=stream)
            torch.cuda.synchronize()
            kms = inst.fista_step(steps, timed=True, stream=stream)
            inst.fista_end(stream=stream, allow=(4, 5))
            it_ms = (kms[0] + kms[1]) / steps
            rows.append({"storage": "matrix-free" if mf else "stored", "log2n": k, "nnz": nnz,
                         "device_bytes": inst.info["device_bytes"], "iteration_ms": it_ms,
                         "gbs": (k1b + k2b) / (it_ms * 1e-3) / 1e9,
                         "frac": (k1b + k2b) / (it_ms * 1e-3) / 1e9 / peak})
            inst.free()
    ctx.close()
    return {"workload": "c2 recipe (m = 2n, ~8/col, FP32 values) at n = 2^k", "peak_gbs": peak, "runs": rows}


def c1_form(l1, W):
    """C1 (m = 2048, n = 1024, FP64, tol 1e-8): the latency-bound case.  FISTA through
    l1ls_solve_fista (CUDA graphs of 32 iterations between host checks) against the same
    iterations launched one kernel at a time (l1ls_fista_begin / step / end), and pdNCG."""
    import torch
    ctx = l1.Context(0)
    inst = ctx.generate(W.C1)
    out = {"workload": "c1: m=2048, n=1024, kappa 1e2, x* 5%, FP64 values, tau=1, gap 1e-8"}
    for rep in range(2):          # the first round warms up (module load, graph build)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, r = inst.solve_fista(tau=1.0, tol=W.C1_TOL, max_iter=200000)
        graph = time.perf_counter() - t
        t = time.perf_counter()
        inst.fista_begin(tau=1.0, tol=W.C1_TOL, max_iter=200000)
        inst.fista_step(r["iters"] + 2)
        _, g = inst.fista_end(allow=(4, 5))
        stepped = time.perf_counter() - t
        t = time.perf_counter()
        _, q = inst.solve_pdncg(tau=1.0, tol=W.C1_TOL, max_iter=200)
        pd = time.perf_counter() - t
    out["fista_graphs"] = {"seconds": graph, "iters": r["iters"], "us_per_iter": 1e6 * graph / r["iters"],
                           "rel_gap": r["rel_gap"], "status": r["status_name"]}
    out["fista_kernel_by_kernel"] = {"seconds": stepped, "iters": g["iters"],
                                     "us_per_iter": 1e6 * stepped / max(g["iters"], 1), "rel_gap": g["rel_gap"],
                                     "status": g["status_name"]}
    out["pdncg"] = {"seconds": pd, "iters": q["iters"], "cg_iters": q["cg_iters"], "rel_gap": q["rel_gap"],
                    "status": q["status_name"]}
    inst.free()
    ctx.close()
    return out


def precision_form(l1, W, limit_s):
    """C3: A stored as FP64 / FP32 / BF16 at kappa 1e2, 1e4, 1e6 (m = 2^22, n = 2^21, 16 per
    column, x* 2%, tau = tau_gen = 1): FISTA (gradient restart; float-float products for FP32 /
    BF16) and pdNCG (float-float gradient products for FP32 / BF16), each to a 1e-6 gap (1e-4 for
    BF16) within `limit_s`, against the FP64 optimum x*, f* of the generator."""
    import numpy as np
    ctx = l1.Context(0)
    rows = []
    for kappa in (1e2, 1e4, 1e6):
        for dt in ("f64", "f32", "bf16"):
            inst = ctx.generate(W.c3(kappa, dt))
            xs = inst.xstar()
            tol = 1e-4 if dt == "bf16" else 1e-6
            f_star = inst.info["f_star"]
            for method in ("fista", "pdncg"):
                t = time.perf_counter()
                if method == "fista":
                    x, r = inst.solve_fista(tau=1.0, tol=tol, max_iter=10 ** 6, restart=1,
                                            accum=0 if dt == "f64" else 1, time_limit_s=limit_s, allow=(4, 5))
                else:
                    x, r = inst.solve_pdncg(tau=1.0, tol=tol, max_iter=200, accum=0 if dt == "f64" else 1,
                                            time_limit_s=limit_s, allow=(4, 5))
                el = time.perf_counter() - t
                rows.append({"kappa": kappa, "values": dt, "method": method, "tol": tol, "status": r["status_name"],
                             "iters": r["iters"], "cg_iters": r["cg_iters"], "seconds": el, "rel_gap": r["rel_gap"],
                             "rel_err_f": abs(r["f"] - f_star) / f_star,
                             "rel_err_x": float(np.linalg.norm(x - xs) / np.linalg.norm(xs))})
            inst.free()
    ctx.close()
    return {"workload": "c3: m=2^22, n=2^21, ~16/col, x* 2%%, tau=1, FISTA with restart and pdNCG, %g s limit "
                        "per solve" % limit_s, "runs": rows}


def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")

    import paper_1503_03520_gb300 as l1
    import workloads as W

    params = rank_workload(args.log2n, rank)
    if args.matrix_free:
        params = dict(params, matrix_free=1)
    ctx = l1.Context(local)
    inst = ctx.generate(params)
    m, n, nnz = inst.m, inst.n, inst.nnz
    k1b, k2b = mf_bytes_per_iteration(m, n) if args.matrix_free else bytes_per_iteration(m, n, nnz)
    k1_name, k2_name = ("k_mf_rt+k_fista_mf1", "k_fista_mf2") if args.matrix_free else ("k_fista_k1", "k_fista_k2")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    # ---- device-timed region: W warm-up + K timed FISTA iterations ---------------------
    inst.fista_begin(tau=1.0, tol=0.0, max_iter=10 ** 12, stream=stream)
    for _ in range(args.warmup):
        inst.fista_step(1, stream=stream)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    kms = inst.fista_step(args.steps, timed=True, stream=stream)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = e0.elapsed_time(e1)
    _, fres = inst.fista_end(stream=stream, allow=(4, 5))
    elapsed_ms = max_over_ranks(elapsed_ms, dist)
    ms_per_step = elapsed_ms / args.steps
    value = (k1b + k2b) * world / (ms_per_step * 1e-3) / 1e9

    # ---- roofline of the dominant kernel --------------------------------------------------
    k1_ms, k2_ms = kms[0] / args.steps, kms[1] / args.steps
    if k2_ms >= k1_ms:
        dom, dom_ms, dom_bytes = k2_name, k2_ms, k2b
    else:
        dom, dom_ms, dom_bytes = k1_name, k1_ms, k1b
    peak, peak_src = measured_hbm_peak()
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src + " (hbm_gbs, copy)",
                "traffic": profiled_traffic(dom), "algorithmic_bytes": dom_bytes,
                "k1_ms": k1_ms, "k2_ms": k2_ms,
                "k1_frac": k1b / (k1_ms * 1e-3) / 1e9 / peak, "k2_frac": k2b / (k2_ms * 1e-3) / 1e9 / peak}

    # ---- e2e through the public API with host buffers -----------------------------------------
    x0 = torch.zeros(n, dtype=torch.float64).pin_memory()
    xo = torch.zeros(n, dtype=torch.float64).pin_memory()
    x0.numpy()[:] = 0.0
    e2e_times = []
    for i in range(args.warmup + args.e2e_steps):
        barrier()
        t = time.perf_counter()
        _, r = inst.solve_fista(x0=x0, x_out=xo, tau=1.0, tol=0.0, max_iter=E2E_ITERS, check_every=E2E_ITERS,
                                stream=stream, allow=(5,))
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t)
    e2e_s = statistics.median(e2e_times)
    e2e_s = max_over_ranks(e2e_s, dist)
    # warm start from x0 costs one extra product A x0 (matrix, x, y)
    e2e_bytes = E2E_ITERS * (k1b + k2b) + (k1b if args.matrix_free else (nnz // 2) * 12 + (m // 2 + 1) * 4 + n * 4 + m * 4)
    e2e = {"value": e2e_bytes * world / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n, "iters_per_step": E2E_ITERS, "steps": args.e2e_steps,
           "api": "l1ls_solve_fista(x0=pinned host, x_out=pinned host)"}

    # ---- time to the 1e-6 gap (reported beside the metric) --------------------------------
    solves = {}
    if not args.no_solves:
        for method in ("fista", "pdncg"):
            fn = inst.solve_fista if method == "fista" else inst.solve_pdncg
            barrier()
            t = time.perf_counter()
            _, r = fn(tau=1.0, tol=W.C2_TOL, max_iter=200000 if method == "fista" else 200,
                      time_limit_s=args.solve_limit, stream=stream, allow=(4, 5))
            el = time.perf_counter() - t
            solves[method] = {"seconds": el, "iters": r["iters"], "cg_iters": r["cg_iters"],
                              "products": r["products"], "rel_gap": r["rel_gap"], "status": r["status_name"],
                              "rel_err_f": abs(r["f"] - inst.info["f_star"]) / inst.info["f_star"]}
        # pdNCG as the paper runs it: mu = 1e-5 without continuation below it (its smoothing
        # bias, about 0.2 tau mu per zero of x*, puts the certificate's floor near 4e-5 here),
        # to a 1e-4 gap; the paper reports the objective it reaches, here against f*
        barrier()
        t = time.perf_counter()
        _, r = inst.solve_pdncg(tau=1.0, tol=1e-4, max_iter=200, mu_min=1e-5, time_limit_s=args.solve_limit,
                                stream=stream, allow=(4, 5))
        el = time.perf_counter() - t
        # the paper's measure (objective against time): time until the objective's excess over
        # the optimum (f* of the generator) is 1e-3 of its value at x = 0, FISTA and pdNCG (the
        # paper's mu) stopped by f_target.  Relative to f* itself the start is already within
        # about 1e-8 (e dominates b, as the paper notes for its noisy instances, Sec. 8.5), so
        # the excess is resolved only to about 4e-4 of its start by FP32 products.
        f_star = inst.info["f_star"]
        _, r0 = inst.solve_fista(tau=1.0, tol=0.0, max_iter=0, stream=stream, allow=(4, 5))
        target = f_star + 1e-3 * (r0["f"] - f_star)
        for method in ("fista", "pdncg"):
            barrier()
            t0 = time.perf_counter()
            if method == "fista":
                _, q = inst.solve_fista(tau=1.0, tol=0.0, f_target=target, max_iter=200000,
                                        time_limit_s=args.solve_limit, stream=stream, allow=(4, 5))
            else:
                _, q = inst.solve_pdncg(tau=1.0, tol=0.0, f_target=target, max_iter=200, mu_min=1e-5,
                                        time_limit_s=args.solve_limit, stream=stream, allow=(4, 5))
            solves["to_objective_" + method] = {
                "target": "f - f* <= 1e-3 (f(0) - f*)", "seconds": time.perf_counter() - t0, "iters": q["iters"],
                "cg_iters": q["cg_iters"], "products": q["products"], "status": q["status_name"],
                "excess_reduction": (q["f"] - f_star) / (r0["f"] - f_star)}
        solves["pdncg_paper_mu"] = {"tol": 1e-4, "mu": 1e-5, "seconds": el, "iters": r["iters"],
                                    "cg_iters": r["cg_iters"], "products": r["products"], "rel_gap": r["rel_gap"],
                                    "status": r["status_name"],
                                    "rel_err_f": abs(r["f"] - inst.info["f_star"]) / inst.info["f_star"]}
        if not args.matrix_free:
            solves["pdncg"]["pcg_iteration"] = pcg_iteration_timing(inst, m, n, nnz)

    inst.free()
    default_forms = {"batch", "matrix_free", "serve", "fista_variants", "c1", "sec89_matrix_free", "precision"}
    if args.forms is not None:
        chosen = set(f for f in args.forms.split(",") if f)
    else:
        chosen = set() if args.no_forms else set(default_forms)
        if args.no_precision:
            chosen.discard("precision")
        if args.sec89_mf_log2n <= 0:
            chosen.discard("sec89_matrix_free")
        chosen |= {f for f, on in (("size_sweep", args.sweep), ("osgen3", args.osgen3), ("sec89", args.sec89)) if on}
    forms = None
    if rank == 0 and chosen:
        forms = {}
        if "batch" in chosen:
            forms["batch"] = batch_form(l1, W, ctx, args.batch_iters)
    ctx.close()
    if rank == 0 and chosen:
        if "matrix_free" in chosen:
            forms["matrix_free"] = mf_form(l1, W, args.log2n, args.steps, args.warmup, args.solve_limit)
        if "serve" in chosen:
            rates = SERVE_RATES if args.serve_rate is None else (args.serve_rate,)
            forms["serve"] = serve_form(l1, W, args.serve_count, rates, args.serve_log2n, args.serve_slots)
        if "fista_variants" in chosen:
            forms["fista_variants"] = variants_form(l1, W, args.variants_log2n, args.solve_limit)
        if "c1" in chosen:
            forms["c1"] = c1_form(l1, W)
        if "size_sweep" in chosen:
            forms["size_sweep"] = sweep_form(l1, W, range(20, 28), range(24, 30), 20, 3)
        if "osgen3" in chosen:
            forms["osgen3"] = osgen3_form(l1, W, args.osgen3_log2n, args.osgen3_limit)
        if "sec89" in chosen:
            forms["sec89"] = sec89_form(l1, W, args.sec89_log2n, (8, 16, 32))
        if "sec89_matrix_free" in chosen:
            forms["sec89_matrix_free"] = sec89_large_form(
                l1, W, args.sec89_mf_log2n, tuple(int(k) for k in args.sec89_mf_newton.split(",") if k),
                tuple(float(k) for k in args.sec89_mf_tol.split(",") if k))
        if "precision" in chosen:
            forms["precision"] = precision_form(l1, W, args.precision_limit)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            log2n = CPU_SAMPLE_LOG2N
            single = cpu_oracle_iterations(log2n, 1, 0, args.cpu_budget)
            multi = cpu_oracle_all_cores(log2n, 1, single["steps"], 0.0)
            cpu = cpu_baseline_line(single, multi, log2n)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (generator of Sec. 3-6, seeded)",
                "config": {"workload": "c2: m=2^%d, n=2^%d, nnz=%d (~8/col), FP32 values, int32 indices, "
                                       "kappa(A)=1e4, x* 1%%, tau=1, one FISTA iteration per step"
                                       % (args.log2n + 1, args.log2n, nnz),
                           "storage": ("A not assembled: products by its factors (stages of R, Sigma, "
                                       "permutation, left rotations), FP32" if args.matrix_free else
                                       "row-pair CSR and column CSR of P1^T A: one int32 index and two FP32 "
                                       "values per pair of entries"),
                           "l2": "inputs larger than L2 (A is %.2f GB per product)" % (nnz * 6 / 1e9),
                           "parallelism": "replicas (one instance per GPU)" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": (3 if args.matrix_free else 2) * args.steps, "fista_rel_gap_after_steps": fres["rel_gap"],
                "time_to_gap": {"tol": W.C2_TOL, **solves}, "forms": forms}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=24)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-solves", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--solve-limit", type=float, default=30.0)
    ap.add_argument("--no-forms", action="store_true", help="skip every form (the legs beside the metric)")
    ap.add_argument("--forms", default=None,
                    help="run exactly these forms (comma list of batch, matrix_free, serve, fista_variants, c1, "
                         "sec89_matrix_free, precision, size_sweep, osgen3, sec89); default: all but the last three")
    ap.add_argument("--batch-iters", type=int, default=300, help="c4: FISTA iterations per tau at most")
    ap.add_argument("--serve-count", type=int, default=48, help="c5: requests per arrival rate")
    ap.add_argument("--serve-rate", type=float, default=None, help="c5: one arrival rate (default: the sweep "
                                                                   "10, 30, 100, 300, 1000, 2000 per s)")
    ap.add_argument("--serve-log2n", type=int, default=23, help="c5: largest log2 n of a request")
    ap.add_argument("--serve-slots", type=int, default=16, help="c5: serving slots")
    ap.add_argument("--no-precision", action="store_true", help="skip the c3 precision sweep (about 30 s)")
    ap.add_argument("--matrix-free", action="store_true",
                    help="time the iteration on the instance with A not assembled (Algorithms MvPA / MvPAt)")
    ap.add_argument("--precision-limit", type=float, default=6.0, help="c3: time limit per solve (s)")
    ap.add_argument("--variants-log2n", type=int, default=22, help="FISTA variants leg: log2 n")
    ap.add_argument("--sweep", action="store_true", help="add the size sweep (n = 2^20 .. 2^27 stored, "
                                                         "2^24 .. 2^29 matrix-free)")
    ap.add_argument("--osgen3", action="store_true", help="add the Sec. 8.5 OsGen3 leg")
    ap.add_argument("--osgen3-log2n", type=int, default=22)
    ap.add_argument("--osgen3-limit", type=float, default=10.0, help="Sec. 8.5 leg: FISTA time limit (s)")
    ap.add_argument("--sec89", action="store_true", help="add the Sec. 8.9 pdNCG leg")
    ap.add_argument("--sec89-log2n", type=int, default=22)
    ap.add_argument("--sec89-mf-log2n", type=int, default=26,
                    help="Sec. 8.9 shape, matrix-free pdNCG at n = 2^k (0: skip; 29 is the largest, m = 2^30)")
    ap.add_argument("--sec89-mf-newton", default="8,16", help="Newton steps of the matrix-free Sec. 8.9 runs")
    ap.add_argument("--sec89-mf-tol", default="", help="relative gaps the matrix-free Sec. 8.9 instance is also "
                                                       "solved to (comma list; default none)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
