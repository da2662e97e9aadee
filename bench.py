#!/usr/bin/env python
"""Benchmark of the curvature-matrix hot path on one GB300.

Workload: MLP [784, 16, 10] with tanh hidden layer, P = 12730 parameters,
N = 1024 synthetic examples (x ~ U[0,1], uniform one-hot labels over 10
classes, Glorot-uniform weights, zero biases, seed 1).  One step is one pass
of the whole hot path: the OPG (forward, per-example gradients, symmetric
rank-N update), the exact Hessian (batched R-operator over blocks of unit
directions and its contraction) and the top-32 OPG eigenpairs (FP64 Gram
matrix, Lanczos, back-projection).

metric: exact-Hessian & OPG entries/s = 2 P^2 delivered entries per step over
the step time.  The plain FP64 path on the same GPU is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P]
  python bench.py --impl reference ...   (the FP64 CPU oracle, timed on the
                                          host cores on a bounded sample)
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "exact-Hessian & OPG entries/s"
UNIT = "entries/s"
WORKLOAD = "mlp_784_16_10"
K_EIG = 32
# workload -> (calls in one step, k of the eigenpairs)
WORKLOADS = {
    "mlp_784_16_10": (("opg", "hessian", "eig"), 32),
    # the precision workload: OPG in BF16 / split-BF16 and the top-100 eigenpairs
    "mlp_1024_64_64_10": (("opg", "eig"), 100),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "fp32", "bf16", "bf16x3"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only", default=None, choices=["opg", "hessian", "eig"],
                    help="run one call of the step (for profiling); the line is then partial")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--serve", action="store_true",
                    help="serving benchmark: Poisson request stream through the request server")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--batch", action="store_true",
                    help="the many-networks workload: OPG + exact Hessian of 256 networks in waves")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--step", default="fused", choices=["fused", "streams", "calls"],
                    help="fused: one hess_curvature call (two internal streams); streams: the "
                         "single calls on two handles and streams; calls: the single calls in turn")
    ap.add_argument("--row", default=None, choices=["hessian-eig", "approx", "minibatch", "stream-eig", "lowmem-eig"],
                    help="hessian-eig: top-k Hessian eigenpairs by Lanczos on H v products; "
                         "approx: low/full-rank approximations from them (own JSON lines)")
    ap.add_argument("--row-k", type=int, default=32)
    ap.add_argument("--lowmem-n", type=int, default=262144)
    ap.add_argument("--lowmem-k", type=int, default=100)
    ap.add_argument("--lowmem-block", type=int, default=0)
    ap.add_argument("--batch-graphs", action="store_true",
                    help="replay each group of the batch from a CUDA graph (use --warmup >= 2)")
    ap.add_argument("--autotune", action="store_true",
                    help="tune the tensor-core tile widths during the warm-up steps")
    ap.add_argument("--batch-workspace-gb", type=float, default=64.0)
    ap.add_argument("--batch-out-gb", type=float, default=96.0)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg of the default line")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the precision workload's OPG leg of the default line")
    ap.add_argument("--serve-leg-seconds", type=float, default=3.0)
    ap.add_argument("--eig-blocks", type=int, default=0,
                    help="most blocks of the eigen step's Lanczos kernel (0: one per SM)")
    ap.add_argument("--probe-fp64", action="store_true",
                    help="measure the FP64 FMA issue rate of the GPU and exit")
    ap.add_argument("--cpu-worker", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


# ------------------------------------------------------------- CPU oracle ----
def cpu_worker(sample_cols: int) -> dict:
    """Runs in a fresh process: the FP64 oracle on a bounded sample of the
    workload -- `sample_cols` Hessian columns (one Hessian-vector product
    each) and the same OPG columns -- timed on the host cores."""
    import numpy as np

    from oracle import mlp as O
    from synth import named_config

    pb = named_config(WORKLOAD)
    rng = np.random.default_rng(0)
    cols = np.sort(rng.choice(pb.P, size=sample_cols, replace=False))
    t0 = time.perf_counter()
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    opg_cols = (G.T @ G[:, cols]) / pb.N
    Hc = O.hessian_columns(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, cols)
    dt = time.perf_counter() - t0
    entries = opg_cols.size + Hc.size
    return {"value": entries / dt, "seconds": dt, "entries": int(entries),
            "sample": f"{sample_cols} Hessian columns (unit-vector HVPs) + {sample_cols} OPG "
                      f"columns of the {WORKLOAD} workload, N={pb.N}, FP64 numpy",
            "cores": os.cpu_count()}


def run_cpu_baseline(sample_cols: int) -> dict:
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker",
                        str(sample_cols)], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def workload_desc(name):
    """The workload string of the bench line (shared by both arms)."""
    from synth import named_config
    pb = named_config(name)
    calls, k = WORKLOADS[name]
    what = " + ".join({"opg": "OPG", "hessian": "exact Hessian", "eig": f"top-{k} OPG eig"}[c] for c in calls)
    return (f"{name}: MLP {pb.widths} {'/'.join(pb.acts)}, P={pb.P}, N={pb.N}; {what} per step",
            pb.P, pb.N, k)


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = []
    for _ in range(args.warmup):
        run_cpu_baseline(64)
    for _ in range(args.steps):
        res.append(run_cpu_baseline(256))
    vals = [r["value"] for r in res if "value" in r]
    secs = [r["seconds"] for r in res if "seconds" in r]
    value = statistics.median(vals) if vals else None
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(secs) if secs else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(zip(("workload", "P", "N", "k"), workload_desc(WORKLOAD)),
                       step="FP64 oracle on the host cores, a bounded sample of the step's "
                            "Hessian and OPG columns per step"),
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle",
                         "cores": res[0].get("cores") if res else None,
                         "sample": res[0].get("sample") if res else None},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu_index), "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and ids[local_rank % len(ids)].strip().isdigit():
        return int(ids[local_rank % len(ids)])
    return local_rank


# --------------------------------------------------------------- serving ----
def serve_leg(seconds, rate, slots, torch=None):
    """Poisson arrivals (seed 4) of exact-Hessian, OPG and top-32 eigenpair
    requests, uniform over the three kinds and over 16 networks of the
    batching distribution, through the continuous-batching request server
    with a 100 GB workspace budget.  Latency = submit to completion (host
    clock); each request's device interval comes from the server's events on
    its slot stream, and the fraction of device-busy time during which two or
    more requests were on the GPU shows the overlap."""
    import threading

    import numpy as np
    if torch is None:
        import torch

    import paper_1905_05559_gb300 as hm
    from synth import SplitMix64Stream, make_problem, make_random_mlp

    nets = []
    for i in range(16):
        widths, acts, N = make_random_mlp(4, i)
        pb = make_problem(widths, acts, N, 400 + i, "normal", "zero")
        nets.append((pb, torch.as_tensor(pb.X, dtype=torch.float32, device="cuda"),
                     torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")))
    srv = hm.HessServer(slots=slots, budget_bytes=100 * (1 << 30))
    ids = [srv.add_network(pb.widths, pb.acts, pb.omega) for pb, _, _ in nets]
    rs = SplitMix64Stream(4, 1)
    n_req = int(rate * seconds)
    gaps = -np.log(1.0 - rs.uniform(n_req)) / rate
    arrivals = np.cumsum(gaps)
    kinds = rs.integers(n_req, 0, 2)
    which = rs.integers(n_req, 0, len(nets) - 1)
    # warm-up: one request of each kind on each network
    for i, (pb, X, Y) in enumerate(nets):
        for kind in ("hessian", "opg", "eig"):
            if kind == "eig":
                out = torch.empty((32, pb.P), dtype=torch.float64, device="cuda")
                ev = torch.empty(32, dtype=torch.float64, device="cuda")
                srv.wait(srv.submit(kind, ids[i], X, Y, "fp32", out, k=32, evals=ev))
            else:
                out = torch.empty((pb.P, pb.P), device="cuda")
                srv.wait(srv.submit(kind, ids[i], X, Y, "bf16x3", out))
    torch.cuda.synchronize()
    lat = [None] * n_req
    dev = [None] * n_req
    entries = [0.0] * n_req
    sem = threading.Semaphore(64)  # the client keeps at most 64 requests in flight
    lock = threading.Lock()
    pending = []

    failures = {}

    def waiter(j, ticket, t_submit, keep):
        st, g0, g1 = srv.wait_timed(ticket)
        t_done = time.perf_counter()
        msg = hm.last_error() if st not in (0, 4) else ""
        with lock:
            lat[j] = (t_done - t_submit, st)
            dev[j] = (g0, g1)
            if msg:
                failures.setdefault(f"{st}: {msg[:120]}", 0)
                failures[f"{st}: {msg[:120]}"] += 1
        del keep
        sem.release()

    t0 = time.perf_counter()
    for j in range(n_req):
        now = time.perf_counter() - t0
        if arrivals[j] > now:
            time.sleep(arrivals[j] - now)
        sem.acquire()
        pb, X, Y = nets[which[j]]
        kind = ("hessian", "opg", "eig")[kinds[j]]
        t_sub = time.perf_counter()
        if kind == "eig":
            out = torch.empty((32, pb.P), dtype=torch.float64, device="cuda")
            ev = torch.empty(32, dtype=torch.float64, device="cuda")
            tk = srv.submit(kind, ids[which[j]], X, Y, "fp32", out, k=32, evals=ev)
            keep = (out, ev)
            entries[j] = 32.0 * pb.P
        else:
            out = torch.empty((pb.P, pb.P), device="cuda")
            tk = srv.submit(kind, ids[which[j]], X, Y, "bf16x3", out)
            keep = (out,)
            entries[j] = float(pb.P) * pb.P
        th = threading.Thread(target=waiter, args=(j, tk, t_sub, keep))
        th.start()
        pending.append(th)
    for th in pending:
        th.join()
    wall = time.perf_counter() - t0
    srv.close()
    ok = [l for l, st in lat if st in (0, 4)]
    ls = np.sort(np.asarray(ok)) * 1e3
    # device concurrency: sweep over the requests' device intervals
    ev = []
    for d in dev:
        if d and d[0] >= 0 and d[1] >= d[0]:
            ev.append((d[0], 1))
            ev.append((d[1], -1))
    ev.sort()
    busy = over = 0.0
    act = 0
    for (t, dlt), (t2, _) in zip(ev, ev[1:] + [(ev[-1][0] if ev else 0.0, 0)]):
        act += dlt
        if act >= 1:
            busy += t2 - t
        if act >= 2:
            over += t2 - t
    spans = sum(d[1] - d[0] for d in dev if d and d[0] >= 0 and d[1] >= d[0])
    return {
        "p50_ms": float(np.percentile(ls, 50)), "p99_ms": float(np.percentile(ls, 99)),
        "entries_per_s": float(sum(entries) / wall), "submitted": n_req, "completed": len(ok),
        "failures": failures, "wall_s": wall, "offered_rate": rate, "achieved_rate": n_req / wall,
        "device_busy_s": busy * 1e-3, "overlap_frac": (over / busy) if busy > 0 else None,
        "mean_concurrency": (spans / busy) if busy > 0 else None, "slots": slots, "seconds": seconds,
        "workload": "Poisson request stream (seed 4): exact Hessian (split-BF16), OPG (split-BF16), "
                    "top-32 OPG eig (FP64 Gram), 16 networks of the batching distribution, "
                    "100 GB workspace budget",
    }


def serve_bench(args):
    import torch
    from paper_1905_05559_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    r = serve_leg(args.serve_seconds, args.serve_rate, args.serve_slots, torch)
    line = {
        "metric": "served p50/p99 latency (ms) and delivered entries/s", "impl": "ours",
        "value": r["p50_ms"], "unit": "ms (p50)", "higher_is_better": False, "n_gpus": 1,
        **{k: v for k, v in r.items() if k != "workload"},
        "config": {"workload": r["workload"], "slots": args.serve_slots, "seconds": args.serve_seconds},
        "data": "synthetic",
    }
    print(json.dumps(line), flush=True)


def precision_leg(hm, torch, peaks):
    """The precision workload's OPG: MLP [1024, 64, 64, 10] ReLU, P = 70410,
    N = 8192, split-BF16 and BF16 on the tensor cores (one warm call, then one
    timed call each); the SYRK's flops over its own CUDA-event time."""
    from synth import named_config
    pb = named_config("mlp_1024_64_64_10")
    P, N = pb.P, pb.N
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    OPG = torch.empty((P, P), dtype=torch.float32, device="cuda")
    out = {"workload": f"mlp_1024_64_64_10: MLP {pb.widths} relu, P={P}, N={N}; one OPG call",
           "P": P, "N": N}
    st = torch.cuda.current_stream()
    for prec, mult in (("bf16x3", 3.0), ("bf16", 1.0)):
        net.opg(X, Y, prec, out=OPG)
        torch.cuda.synchronize()
        net.read_timing("syrk")
        net.timing(True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        net.opg(X, Y, prec, out=OPG)
        b.record(st)
        torch.cuda.synchronize()
        net.timing(False)
        k = net.read_timing("syrk")
        call_ms = a.elapsed_time(b)
        tf = mult * k["flops"] / (k["ms"] * 1e-3) / 1e12 if k["ms"] > 0 else None
        out[prec] = {"call_ms": call_ms, "opg_entries_per_s": float(P) * P / (call_ms * 1e-3),
                     "syrk_ms": k["ms"], "syrk_tflops": tf,
                     "syrk_frac": tf / peaks["bf16_tflops_sustained"] if tf else None,
                     "peak": peaks["bf16_tflops_sustained"], "peak_source": "measured bf16 sustained"}
    del OPG
    net.close()
    torch.cuda.empty_cache()
    return out


def batch_bench(args):
    """The many-networks workload: networks 0..count-1 of the batching
    distribution (seed 3; 2-4 weight layers, P in [500, 20000], N in
    [64, 2048]), the OPG and the exact Hessian of each in split-BF16 through
    hess_batch_run.  The outputs of all 256 networks (~273 GB in FP32) do not
    fit in HBM, so a step runs the list in groups whose outputs fit an output
    pool; inside a group the batch forms waves of one persistent tensor-core
    launch each.  Every finished matrix is checked outside the timed region
    (finite, sampled symmetry, trace(OPG) = ||G||_F^2 / N with G from
    per_example_grads) before its memory is reused by the next group."""
    import numpy as np
    import torch

    import paper_1905_05559_gb300 as hm
    from paper_1905_05559_gb300 import build
    from synth.inputs import make_batch_problem

    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    lib = hm.load()
    pbs = [make_batch_problem(3, i) for i in range(args.batch_count)]
    nets = [hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=stream.cuda_stream) for pb in pbs]
    Xs = [torch.as_tensor(pb.X, dtype=torch.float32, device="cuda") for pb in pbs]
    Ys = [torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda") for pb in pbs]
    pool = torch.empty(int(args.batch_out_gb * (1 << 30)) // 4, dtype=torch.float32, device="cuda")
    groups, cur, used = [], [], 0
    for i, pb in enumerate(pbs):
        need = 2 * ((pb.P * pb.P + 63) // 64 * 64)
        if cur and used + need > pool.numel():
            groups.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += need
    groups.append(cur)
    batch = hm.HessBatch(int(args.batch_workspace_gb * (1 << 30)), stream=stream.cuda_stream)
    if args.batch_graphs:
        batch.set_graphs(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rng = np.random.default_rng(3)

    def group_outputs(g):
        off, outs = 0, []
        for i in g:
            P = pbs[i].P
            sz = (P * P + 63) // 64 * 64
            o = pool[off:off + P * P].view(P, P)
            off += sz
            h = pool[off:off + P * P].view(P, P)
            off += sz
            outs.append((o, h))
        return outs

    def check(i, o, h):
        pb = pbs[i]
        assert bool(torch.isfinite(o).all()) and bool(torch.isfinite(h).all()), i
        r = torch.as_tensor(rng.choice(pb.P, size=min(64, pb.P), replace=False), device="cuda")
        c = torch.as_tensor(rng.choice(pb.P, size=min(64, pb.P), replace=False), device="cuda")
        for m in (o, h):
            assert torch.equal(m[r][:, c], m[c][:, r].T), i
        G = nets[i].per_example_grads(Xs[i], Ys[i], "fp32")
        tr = float((G.double() ** 2).sum()) / pb.N
        rel = abs(float(torch.trace(o.double())) - tr) / tr
        # split-BF16 drops the lo*lo term, a bias of about 2^-16 / 3 on
        # diagonal entries: a loose sanity bound here, parity is in the tests
        assert rel <= 3e-5, (i, rel)
        return rel

    def one_pass(do_check):
        ms = launch_ms = flops = 0.0
        waves = chunked = replayed = 0
        worst = 0.0
        for g in groups:
            outs = group_outputs(g)
            items = [(nets[i], Xs[i], Ys[i], o, h) for i, (o, h) in zip(g, outs)]
            torch.cuda.synchronize()
            ev0.record(stream)
            info = batch.run(items, "bf16x3")
            ev1.record(stream)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
            launch_ms += info["launch_ms"]
            flops += info["flops"]
            waves += info["waves"]
            chunked += info["items_chunked"]
            replayed += int(info["graph_replayed"])
            if do_check:
                for i, (o, h) in zip(g, outs):
                    worst = max(worst, check(i, o, h))
        return ms, launch_ms, flops, waves, chunked, worst, replayed

    if args.autotune:
        hm.autotune(True)
    for _ in range(args.warmup):
        one_pass(False)
    hm.autotune(False)
    sampler = ClockSampler(gpu_index(0))
    sampler.start()
    l0 = lib.hess_launch_count()
    runs = [one_pass(True) for _ in range(args.steps)]
    launches = (lib.hess_launch_count() - l0) / args.steps
    clocks = sampler.stop()
    ms = statistics.median(r[0] for r in runs)
    launch_ms = statistics.median(r[1] for r in runs)
    flops, waves, chunked = runs[0][2], runs[0][3], runs[0][4]
    entries = float(sum(2.0 * pb.P * pb.P for pb in pbs))
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained") or 1700.0
    achieved = flops / (launch_ms * 1e-3) / 1e12
    line = {
        "metric": "exact-Hessian & OPG entries/s (many networks)", "impl": "ours",
        "value": entries / (ms * 1e-3), "unit": "entries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3",
        "data": "synthetic",
        "config": {"workload": f"{args.batch_count} MLPs of the batching distribution (seed 3), "
                               "OPG + exact Hessian each, split-BF16",
                   "networks": args.batch_count, "groups": len(groups), "waves": waves,
                   "tile_widths": (f"autotuned ({hm.autotune_entries()} shapes)" if args.autotune
                                   else "cost model"),
                   "cuda_graphs": (f"{runs[-1][6]} of {len(groups)} groups replayed" if args.batch_graphs
                                   else "off"),
                   "items_alone": chunked,
                   "workspace_gb": args.batch_workspace_gb, "output_pool_gb": args.batch_out_gb,
                   "l2": "outputs and operands far larger than L2"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel_class": "wave launches",
                     "peak_source": f"{src} bf16 sustained",
                     "note": "split-BF16 counts three BF16 products per multiply-add"},
        "launch_ms_per_step": launch_ms, "prep_ms_per_step": ms - launch_ms,
        "max_trace_rel": max(r[5] for r in runs), "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    batch.close()



def heig_bench(args):
    """Top-k eigenpairs of the exact Hessian by Lanczos on the operator
    v -> H v (hessian_topk_eig), never forming H: the MLP workload (P = 12730,
    N = 1024), k = 32, FP64 products and recurrence.  One step = one solve.
    The CPU baseline is the oracle's route (all P Hessian columns from its
    products, then a dense eigensolver), timed on a sample: 256 columns and
    the eigensolver on a 3072 x 3072 symmetric matrix, scaled by P / 256 and
    (P / 3072)^3."""
    import numpy as np
    import torch

    import paper_1905_05559_gb300 as hm
    from paper_1905_05559_gb300 import build
    from synth import named_config

    cpu = None
    if not args.no_cpu_baseline:
        from oracle import mlp as O
        pb = named_config(args.workload)
        t0 = time.perf_counter()
        O.hessian_columns(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, range(256))
        t_cols = time.perf_counter() - t0
        A = np.random.default_rng(0).standard_normal((3072, 3072))
        A = A + A.T
        t0 = time.perf_counter()
        np.linalg.eigh(A)
        t_eig = time.perf_counter() - t0
        est = t_cols * pb.P / 256 + t_eig * (pb.P / 3072) ** 3
        cpu = {"value": 1.0 / est, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"256 of {pb.P} Hessian columns ({t_cols:.1f} s) and eigh of 3072^2 "
                         f"({t_eig:.1f} s), scaled to one solve ({est:.0f} s)"}

    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    lib = hm.load()
    pb = named_config(args.workload)
    k = args.row_k
    prec = "fp64" if args.precision not in ("fp32",) else "fp32"
    dt = torch.float64 if prec == "fp64" else torch.float32
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=stream.cuda_stream)
    X = torch.as_tensor(pb.X, dtype=dt, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=dt, device="cuda")
    ev = torch.empty(k, dtype=torch.float64, device="cuda")
    Q = torch.empty((k, pb.P), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    steps = 0
    for _ in range(args.warmup):
        _, _, steps = net.hessian_topk_eig(X, Y, k, prec, evals=ev, evecs=Q)
    torch.cuda.synchronize()
    for cls in ("hvp", "hlanczos"):
        net.read_timing(cls)
    net.timing(True)
    sampler = ClockSampler(gpu_index(0))
    sampler.start()
    l0 = lib.hess_launch_count()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, _, steps = net.hessian_topk_eig(X, Y, k, prec, evals=ev, evecs=Q)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    launches = (lib.hess_launch_count() - l0) / args.steps
    clocks = sampler.stop()
    net.timing(False)
    lz = net.read_timing("hlanczos")
    t = statistics.median(ms)
    peak = 1.25
    achieved = lz["flops"] / (lz["ms"] * 1e-3) / 1e12 if lz["ms"] > 0 else None
    # end to end: host inputs, host outputs
    Xh = np.ascontiguousarray(pb.X, dtype=np.float64 if prec == "fp64" else np.float32)
    Yh = np.ascontiguousarray(pb.Y, dtype=Xh.dtype)
    evh = np.empty(k)
    Qh = np.empty((k, pb.P))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        net.hessian_topk_eig(Xh, Yh, k, prec, evals=evh, evecs=Qh)
    e2e_s = (time.perf_counter() - t0) / args.steps
    line = {
        "metric": f"Hessian top-{k} eigenpair solves/s", "impl": "ours", "value": 1000.0 / t,
        "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32 products, f64 recurrence", "data": "synthetic",
        "config": {"workload": f"{args.workload}: MLP {pb.widths} {'/'.join(pb.acts)}, P={pb.P}, "
                               f"N={pb.N}; top-{k} Hessian eigenpairs, Lanczos on H v",
                   "krylov_dim": steps, "l2": "flushed between solves (256 MiB write)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "kernel_class": "hlanczos (H v products + reorthogonalisation)",
                     "peak_source": "FP64 1.25 TFLOP/s (152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz)",
                     "ms_per_step": lz["ms"] / args.steps, "launches_per_step": lz["launches"] / args.steps},
        "cpu_baseline": cpu,
        "e2e": {"value": 1.0 / e2e_s, "unit": "solves/s",
                "h2d_bytes_per_step": Xh.nbytes + Yh.nbytes, "d2h_bytes_per_step": evh.nbytes + Qh.nbytes},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def approx_bench(args):
    """Low-rank / full-rank approximations (Sec. 4.1, 4.2) from the top-k
    Hessian eigenpairs of the MLP workload: forming the P x P full-rank
    matrix (FP64 and FP32) and applying it implicitly to a block of 1024
    directions (Sec. 5.5, 5.6).  One step = one form in FP32 + one form in
    FP64 + one implicit application."""
    import numpy as np
    import torch

    import paper_1905_05559_gb300 as hm
    from paper_1905_05559_gb300 import build
    from synth import named_config

    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    lib = hm.load()
    pb = named_config(args.workload)
    k = args.row_k
    P = pb.P
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=stream.cuda_stream)
    X = torch.as_tensor(pb.X, dtype=torch.float64, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float64, device="cuda")
    lam, Q, _ = net.hessian_topk_eig(X, Y, k, "fp64")
    b = 1024
    V = torch.as_tensor(np.random.default_rng(0).standard_normal((b, P)), device="cuda")
    out64 = torch.empty((P, P), dtype=torch.float64, device="cuda")
    out32 = torch.empty((P, P), dtype=torch.float32, device="cuda")

    def step():
        net.approx_form(lam, Q, full=True, prec="fp32", out=out32)
        net.approx_form(lam, Q, full=True, prec="fp64", out=out64)
        net.approx_apply(lam, Q, V, full=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    parts = {}
    for name, fn in (("form_fp32", lambda: net.approx_form(lam, Q, full=True, prec="fp32", out=out32)),
                     ("form_fp64", lambda: net.approx_form(lam, Q, full=True, prec="fp64", out=out64)),
                     ("apply_fp64", lambda: net.approx_apply(lam, Q, V, full=True))):
        ts = []
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            e.synchronize()
            ts.append(a.elapsed_time(e))
        parts[name] = statistics.median(ts)
    sampler = ClockSampler(gpu_index(0))
    sampler.start()
    l0 = lib.hess_launch_count()
    ms = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        e.record(stream)
        e.synchronize()
        ms.append(a.elapsed_time(e))
    launches = (lib.hess_launch_count() - l0) / args.steps
    clocks = sampler.stop()
    t = statistics.median(ms)
    peaks, src = measured_peaks()
    f64 = P * (P + 1) * k / (parts["form_fp64"] * 1e-3) / 1e12
    f32 = P * (P + 1) * k / (parts["form_fp32"] * 1e-3) / 1e12
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    app = 4.0 * P * k * b / (parts["apply_fp64"] * 1e-3) / 1e12
    line = {
        "metric": "full-rank approximation entries/s (formed, FP32 + FP64)", "impl": "ours",
        "value": 2.0 * P * P / (t * 1e-3), "unit": "entries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: P={P}, top-{k} Hessian eigenpairs; full-rank form "
                               f"(lam_tilde = lam_K) in FP32 and FP64, implicit application to {b} "
                               "directions", "l2": "outputs (1.9 GB) far larger than L2"},
        "parts_ms": parts,
        "roofline": {"bound": "alu", "achieved": f64, "peak": 1.25, "unit": "TFLOP/s", "frac": f64 / 1.25,
                     "traffic": None, "kernel_class": "approx (FP64 form: upper tiles of Q^T diag(w) Q)",
                     "peak_source": "FP64 1.25 TFLOP/s (152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz)"},
        "rooflines": {
            "form_fp32": {"bound": "alu", "achieved": f32, "peak": fp32_peak, "unit": "TFLOP/s",
                          "frac": f32 / fp32_peak, "hbm_gbs": P * P * 4 / (parts["form_fp32"] * 1e-3) / 1e9,
                          "hbm_peak": peaks["hbm_gbs"]},
            "apply_fp64": {"bound": "alu", "achieved": app, "peak": 1.25, "unit": "TFLOP/s", "frac": app / 1.25}},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def minibatch_bench(args):
    """Mini-batch Hessians (Sec. 5.1) of the MLP workload: the N = 1024
    examples in 16 mini-batches of 64, one P x P split-BF16 Hessian each
    (10.4 GB of output), through the handle's batch waves."""
    import torch

    import paper_1905_05559_gb300 as hm
    from paper_1905_05559_gb300 import build
    from synth import named_config

    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    lib = hm.load()
    pb = named_config(args.workload)
    P, N, bs = pb.P, pb.N, 64
    nb = -(-N // bs)
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=stream.cuda_stream)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    out = torch.empty((nb, P, P), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        net.hessian_minibatches(X, Y, bs, args.precision, out=out)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index(0))
    sampler.start()
    l0 = lib.hess_launch_count()
    ms = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        net.hessian_minibatches(X, Y, bs, args.precision, out=out)
        e.record(stream)
        e.synchronize()
        ms.append(a.elapsed_time(e))
    launches = (lib.hess_launch_count() - l0) / args.steps
    clocks = sampler.stop()
    t = statistics.median(ms)
    line = {
        "metric": "mini-batch Hessian entries/s", "impl": "ours", "value": nb * P * P / (t * 1e-3),
        "unit": "entries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: P={P}, N={N} in {nb} mini-batches of {bs}, one exact "
                               "Hessian each", "l2": "outputs (10.4 GB) far larger than L2"},
        "hbm_write_gbs": nb * P * P * 4 / (t * 1e-3) / 1e9,
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def stream_eig_bench(args):
    """Top-32 OPG eigenpairs of the 784-16-10 tanh network over N = 262144
    seeded examples (the same distribution and seed as the MLP workload, 256x
    the examples; beyond the Gram route's N limit), from chunks of 8192
    examples: split-BF16 chunk OPGs summed into a P x P FP64 matrix, FP64
    Lanczos on it.  metric: examples/s."""
    import torch

    import paper_1905_05559_gb300 as hm
    from paper_1905_05559_gb300 import build
    from synth import make_problem

    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    lib = hm.load()
    N, k, chunk = 262144, args.row_k, 8192
    pb = make_problem([784, 16, 10], ["tanh"], N, 1, "uniform", "zero")
    P = pb.P
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=stream.cuda_stream)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    ev = torch.empty(k, dtype=torch.float64, device="cuda")
    Q = torch.empty((k, P), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        net.opg_topk_eig_streaming(X, Y, k, "bf16x3", chunk=chunk, evals=ev, evecs=Q)
    torch.cuda.synchronize()
    for cls in ("syrk", "eig"):
        net.read_timing(cls)
    net.timing(True)
    sampler = ClockSampler(gpu_index(0))
    sampler.start()
    l0 = lib.hess_launch_count()
    ms = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        net.opg_topk_eig_streaming(X, Y, k, "bf16x3", chunk=chunk, evals=ev, evecs=Q)
        e.record(stream)
        e.synchronize()
        ms.append(a.elapsed_time(e))
    launches = (lib.hess_launch_count() - l0) / args.steps
    clocks = sampler.stop()
    net.timing(False)
    syrk = net.read_timing("syrk")
    eig = net.read_timing("eig")
    t = statistics.median(ms)
    peaks, src = measured_peaks()
    achieved = 3.0 * syrk["flops"] / (syrk["ms"] * 1e-3) / 1e12 if syrk["ms"] > 0 else None
    peak = peaks["bf16_tflops_sustained"]
    line = {
        "metric": f"examples/s (top-{k} OPG eigenpairs, streamed)", "impl": "ours", "value": N / (t * 1e-3),
        "unit": "examples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 (OPG), f64 (eig)",
        "data": "synthetic",
        "config": {"workload": f"MLP [784, 16, 10] tanh, P={P}, N={N} (seed 1, x ~ U[0,1)), chunks of {chunk}; "
                               f"top-{k} OPG eigenpairs", "l2": "inputs (822 MB) larger than L2"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "kernel_class": "syrk (chunk OPGs)", "peak_source": f"{src} bf16 sustained",
                     "ms_per_step": syrk["ms"] / args.steps},
        "eig_ms_per_step": eig["ms"] / args.steps,
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def lowmem_eig_bench(args):
    """Top-k OPG eigenpairs in O(k P) memory (opg_topk_eig_lowmem): the
    precision workload's network (MLP [1024, 64, 64, 10] ReLU, P = 70410)
    over N = 262144 seeded examples (x ~ N(0,1), seed 2), chunks of 8192, FP32
    products, FP64 basis; neither G, nor the Gram matrix, nor the 8 P^2-byte
    OPG is formed.  metric: examples/s; the device memory the call holds is
    reported beside the P x P route's."""
    import ctypes

    import torch

    import paper_1905_05559_gb300 as hm
    from paper_1905_05559_gb300 import _lib, build
    from synth import named_config

    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    lib = hm.load()
    N, k, chunk = args.lowmem_n, args.lowmem_k, 8192
    pb = named_config("mlp_1024_64_64_10", N=N)
    P = pb.P
    free0, total = torch.cuda.mem_get_info()
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=stream.cuda_stream)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    ev = torch.empty(k, dtype=torch.float64, device="cuda")
    Q = torch.empty((k, P), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free_in, _ = torch.cuda.mem_get_info()
    passes = ctypes.c_int()

    def call():
        st = lib.opg_topk_eig_lowmem(net.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), N, k,
                                     _lib.PRECISION["fp32"], chunk, args.lowmem_block,
                                     ctypes.c_void_p(ev.data_ptr()), ctypes.c_void_p(Q.data_ptr()),
                                     ctypes.byref(passes))
        _lib.check(st, allow=(_lib.HESS_ERR_RANK_DEFICIENT,))

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    free_ws, _ = torch.cuda.mem_get_info()
    for c in ("lowmem", "lanczos", "tridiag", "gram", "backproj", "eig"):
        net.read_timing(c)
    net.timing(True)
    sampler = ClockSampler(gpu_index(0))
    sampler.start()
    l0 = lib.hess_launch_count()
    ms = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        e.record(stream)
        e.synchronize()
        ms.append(a.elapsed_time(e))
    launches = (lib.hess_launch_count() - l0) / args.steps
    clocks = sampler.stop()
    net.timing(False)
    lm = net.read_timing("lowmem")
    other = {c: net.read_timing(c)["ms"] / args.steps for c in ("lanczos", "tridiag", "gram", "backproj", "eig")}
    t = statistics.median(ms)
    smx = measured_peaks()[0].get("sm_max_mhz", 2070.0) * 1e6
    fp32_peak = 152 * 128 * 2 * smx / 1e12
    achieved = lm["flops"] / (lm["ms"] * 1e-3) / 1e12 if lm["ms"] > 0 else None
    line = {
        "metric": f"examples/s (top-{k} OPG eigenpairs, O(kP) memory)", "impl": "ours", "value": N / (t * 1e-3),
        "unit": "examples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (products), f64 (basis)",
        "data": "synthetic",
        "config": {"workload": f"MLP {pb.widths} relu, P={P}, N={N} (seed 2, x ~ N(0,1)), chunks of {chunk}; "
                               f"top-{k} OPG eigenpairs", "l2": f"inputs ({X.numel() * 4 / 1e9:.2f} GB) larger than L2"},
        "passes": passes.value,
        "device_bytes": {"inputs": free0 - free_in, "workspace": free_in - free_ws,
                         "pxp_route_opg_alone": 8 * P * P},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak if achieved else None, "traffic": None,
                     "kernel_class": "lowmem (passes over the data: 4 N P b flops each, and the basis updates)",
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock",
                     "ms_per_step": lm["ms"] / args.steps},
        "evals_head": [float(v) for v in ev[:4].cpu()],
        "projected_eig_ms_per_step": other,
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- replicas ----
def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """Replicas only: every rank runs the whole workload on its own GPU and
    the job's time is the slowest rank's (no collective on the data path)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(entries_per_rank: float, step_seconds_max: float, world: int) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return world * entries_per_rank / step_seconds_max


# ------------------------------------------------------------------ GPU ----
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def fp64_probe(lib, torch, iters=10000):
    """The FP64 issue rate of this GPU, measured now: hess_probe_fp64 runs
    eight independent FMA chains per thread over 4 x 256 threads per SM; its
    flops over its CUDA-event duration (one warm-up launch first)."""
    import ctypes
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    fl = ctypes.c_double()
    lib.hess_probe_fp64(200, ctypes.byref(fl), ctypes.c_void_p(sink.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    lib.hess_probe_fp64(iters, ctypes.byref(fl), ctypes.c_void_p(sink.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    return {"tflops": fl.value / (ms * 1e-3) / 1e12, "ms": ms, "flops": fl.value}


def probe_main(args):
    """--probe-fp64: the FP64 issue rate with the SM clock sampled during a
    longer run of the same probe kernel."""
    import torch
    from paper_1905_05559_gb300 import build
    build.build()
    import paper_1905_05559_gb300 as hm
    lib = hm.load()
    fp64_probe(lib, torch, 1000)
    sampler = ClockSampler(gpu_index(0))
    sampler.start()
    runs = [fp64_probe(lib, torch, 50000) for _ in range(5)]
    clocks = sampler.stop()
    best = max(r["tflops"] for r in runs)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = {"probe": "fp64_probe_kernel", "tflops_best": best, "tflops_runs": [r["tflops"] for r in runs],
           "ms_per_run": [r["ms"] for r in runs], "sms": sms, "clocks": clocks}
    if clocks and clocks.get("sm_mhz"):
        out["fp64_fma_per_clk_per_sm"] = best * 1e12 / 2.0 / (clocks["sm_mhz"] * 1e6) / sms
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.cpu_worker:
        print(json.dumps(cpu_worker(args.cpu_worker)), flush=True)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.probe_fp64:
        probe_main(args)
        return
    if args.serve:
        serve_bench(args)
        return
    if args.batch:
        batch_bench(args)
        return
    if args.row == "hessian-eig":
        heig_bench(args)
        return
    if args.row == "approx":
        approx_bench(args)
        return
    if args.row == "minibatch":
        minibatch_bench(args)
        return
    if args.row == "stream-eig":
        stream_eig_bench(args)
        return
    if args.row == "lowmem-eig":
        lowmem_eig_bench(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    # the CPU baseline runs first, in a fresh process, before this process
    # uses the GPU heavily (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        cpu = run_cpu_baseline(2048)

    from paper_1905_05559_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    import paper_1905_05559_gb300 as hm
    from synth import named_config

    calls, K_EIG_W = WORKLOADS[args.workload]
    if args.only:
        calls = tuple(c for c in calls if c == args.only)
    pb = named_config(args.workload)
    P, N = pb.P, pb.N
    stream = torch.cuda.current_stream()
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=stream.cuda_stream)
    if args.eig_blocks:
        net.set_eig_blocks(args.eig_blocks)
    lib = hm.load()
    # two streams: OPG + H on one handle, the eigenpairs on another (each
    # handle owns its workspace); the FP64 Gram work overlaps the tensor-core
    # contractions
    fused = args.step == "fused" and "eig" in calls and len(calls) > 1
    two = args.step == "streams" and "eig" in calls and len(calls) > 1
    if two:
        # the eigen stream has the higher priority: when SMs free up its
        # cooperative Lanczos launch is placed before further contraction CTAs
        s_mat, s_eig = torch.cuda.Stream(priority=0), torch.cuda.Stream(priority=-1)
        net_m = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=s_mat.cuda_stream)
        net_e = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=s_eig.cuda_stream)
        handles = (net_m, net_e)
    else:
        net_m = net_e = net
        handles = (net,)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()

    def make_io(prec):
        dt = torch.float64 if prec == "fp64" else torch.float32
        X = torch.as_tensor(pb.X, dtype=dt, device="cuda")
        Y = torch.as_tensor(pb.Y, dtype=dt, device="cuda")
        H = torch.empty((P, P), dtype=dt, device="cuda") if "hessian" in calls else None
        OPG = torch.empty((P, P), dtype=dt, device="cuda") if "opg" in calls else None
        ev = torch.empty(K_EIG_W, dtype=torch.float64, device="cuda")
        Q = torch.empty((K_EIG_W, P), dtype=torch.float64, device="cuda")
        return X, Y, H, OPG, ev, Q

    def step(prec, io):
        X, Y, H, OPG, ev, Q = io
        if fused:
            net.curvature(X, Y, prec, opg=OPG, hessian=H, k=K_EIG_W, evals=ev, evecs=Q)
            return
        if two:
            start = torch.cuda.Event()
            start.record(stream)
            s_mat.wait_event(start)
            s_eig.wait_event(start)
        if "opg" in calls:
            net_m.opg(X, Y, prec, out=OPG)
        if "hessian" in calls:
            net_m.exact_hessian(X, Y, prec, out=H)
        if "eig" in calls:
            net_e.opg_topk_eig(X, Y, K_EIG_W, prec, evals=ev, evecs=Q)
        if two:
            for st in (s_mat, s_eig):
                done = torch.cuda.Event()
                done.record(st)
                stream.wait_event(done)

    def timed(prec, steps, warmup, sampler=None):
        io = make_io(prec)
        if args.autotune:
            hm.autotune(True)
        for _ in range(warmup):
            step(prec, io)
        hm.autotune(False)
        torch.cuda.synchronize()
        for hd in handles:
            for cls in hm._lib.KERNEL_CLASS:
                hd.read_timing(cls)
            hd.timing(True)
        l0 = lib.hess_launch_count()
        if sampler:
            sampler.start()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ms = []
        for _ in range(steps):
            flush.zero_()  # evicts L2 (256 MiB > 129 MB); outside the events
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(prec, io)
            b.record(stream)
            ms.append((a, b))
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
        clocks = sampler.stop() if sampler else None
        launches = lib.hess_launch_count() - l0
        kern = {}
        for hd in handles:
            hd.timing(False)
            for cls in hm._lib.KERNEL_CLASS:
                r = hd.read_timing(cls)
                acc = kern.setdefault(cls, {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0, "sm_ms": 0.0})
                for kk in acc:
                    acc[kk] += r[kk]
        per = [x.elapsed_time(y) for x, y in ms]
        t = max_over_ranks(sum(per) / len(per), dist if world > 1 else None, "cuda")
        del io
        return t, wall, launches, kern, clocks

    sampler = ClockSampler(gpu_index(local_rank)) if rank == 0 else None
    ms_step, wall, launches, kern, clocks = timed(args.precision, args.steps, args.warmup, sampler)
    entries = float(P) * P * sum(1 for c in calls if c in ("opg", "hessian"))
    value = job_throughput(entries, ms_step * 1e-3, world)

    fp64 = None
    if not args.no_fp64 and args.precision != "fp64":
        ms64, _, _, kern64, _ = timed("fp64", args.fp64_steps, 1)
        fp64 = {"value": job_throughput(entries, ms64 * 1e-3, world), "ms_per_step": ms64,
                "kernels_ms_per_step": {k: v["ms"] / max(args.fp64_steps, 1) for k, v in kern64.items()}}

    # end to end through the C ABI with host buffers: the library stages the
    # pinned host inputs to the device and the outputs back every step
    e2e = None
    if not args.no_e2e:
        npdt = np.float64 if args.precision == "fp64" else np.float32
        pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()  # noqa: E731
        tdt = torch.float64 if args.precision == "fp64" else torch.float32
        Xh = pin(pb.X.shape, tdt)
        Xh[:] = pb.X.astype(npdt)
        Yh = pin(pb.Y.shape, tdt)
        Yh[:] = pb.Y.astype(npdt)
        Hh = pin((P, P), tdt) if "hessian" in calls else None
        Oh = pin((P, P), tdt) if "opg" in calls else None
        evh = pin((K_EIG_W,), torch.float64)
        Qh = pin((K_EIG_W, P), torch.float64)

        if fused:
            def host_step():
                net.curvature(Xh, Yh, args.precision, opg=Oh, hessian=Hh, k=K_EIG_W, evals=evh,
                              evecs=Qh)
        elif two:
            # each call on its own handle, stream and host thread (the calls
            # wait for their own copies; ctypes releases the GIL), so the
            # output copies of one overlap the others' compute
            import threading
            s_o = torch.cuda.Stream()
            net_o = hm.HessMLP(pb.widths, pb.acts, pb.omega, stream=s_o.cuda_stream)
            jobs = []
            if "opg" in calls:
                jobs.append(lambda: net_o.opg(Xh, Yh, args.precision, out=Oh))
            if "hessian" in calls:
                jobs.append(lambda: net_m.exact_hessian(Xh, Yh, args.precision, out=Hh))
            if "eig" in calls:
                jobs.append(lambda: net_e.opg_topk_eig(Xh, Yh, K_EIG_W, args.precision, evals=evh,
                                                       evecs=Qh))

            def host_step():
                errs = []

                def run(f):
                    try:
                        f()
                    except Exception as ex:  # re-raised below
                        errs.append(ex)
                ths = [threading.Thread(target=run, args=(f,)) for f in jobs]
                for t in ths:
                    t.start()
                for t in ths:
                    t.join()
                if errs:
                    raise errs[0]
        else:
            def host_step():
                if "opg" in calls:
                    net.opg(Xh, Yh, args.precision, out=Oh)
                if "hessian" in calls:
                    net.exact_hessian(Xh, Yh, args.precision, out=Hh)
                if "eig" in calls:
                    net.opg_topk_eig(Xh, Yh, K_EIG_W, args.precision, evals=evh, evecs=Qh)

        host_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        torch.cuda.synchronize()
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist if world > 1 else None,
                               "cuda")
        isz = Xh.itemsize
        outs = [a for a in (Hh, Oh) if a is not None]
        e2e = {"value": job_throughput(entries, e2e_s, world), "unit": UNIT,
               "h2d_bytes_per_step": len(calls) * (Xh.size + Yh.size) * isz,
               "d2h_bytes_per_step": sum(a.size for a in outs) * isz
               + ((evh.size + Qh.size) * 8 if "eig" in calls else 0)}

    peaks, peak_src = measured_peaks()
    smx = peaks.get("sm_max_mhz", 2070.0) * 1e6
    fp64_nominal = 1.25  # TFLOP/s: the platform's nominal FP64 rate
    fp32_peak = 152 * 128 * 2 * smx / 1e12
    n_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    probe = fp64_probe(lib, torch) if rank == 0 else None
    bf16_peak = peaks["bf16_tflops_sustained"]
    mult = 3.0 if args.precision == "bf16x3" else 1.0
    # kernel-level classes (one kernel, or one kernel's launches) and what
    # each one is; the composite classes (eig: the whole eigen step; gram,
    # backproj: several small kernels) are reported by time only
    kernel_of = {
        "syrk": "umma_gemm_kernel (OPG contraction)",
        "hcontract": "umma_gemm_kernel (Hessian contraction)",
        "digits": "umma_gemm_kernel (exact-digit FP64 products of the Gram matrix and back-projection)",
        "lanczos": "lanczos kernel on the Gram matrix (cooperative launch)",
        "grads": "write_grads_kernel",
        "tridiag": "bisect_cluster_kernel + inviter_df_kernel",
    }

    def class_roofline(cls):
        k = kern[cls]
        if cls not in kernel_of or k["ms"] <= 0:
            return None
        sec = k["ms"] * 1e-3
        if cls in ("syrk", "hcontract") and args.precision in ("bf16", "bf16x3"):
            r = {"bound": "tensor", "achieved": mult * k["flops"] / sec / 1e12, "peak": bf16_peak,
                 "unit": "TFLOP/s", "peak_source": f"{peak_src} bf16 sustained",
                 "work": f"{mult:g} BF16 products x N P (P+1) (OPG) or the Hessian's contraction flops"}
        elif cls == "digits":
            r = {"bound": "tensor", "achieved": k["flops"] / sec / 1e12, "peak": bf16_peak,
                 "unit": "TFLOP/s", "peak_source": f"{peak_src} bf16 sustained",
                 "work": "BF16 digit-product flops of the exact-digit FP64 products"}
        elif cls == "lanczos":
            pk = probe["tflops"] if probe else fp64_nominal
            r = {"bound": "alu", "achieved": k["flops"] / sec / 1e12, "peak": pk,
                 "unit": "TFLOP/s",
                 "peak_source": ("measured in this run: FP64 FMA issue rate of hess_probe_fp64"
                                 if probe else "FP64 nominal 1.25 TFLOP/s") + " (nominal 1.25)",
                 "work": "sum over Lanczos steps j of 2 N^2 + 8 N (j + 1) FP64-class flops"}
        elif cls == "grads":
            r = {"bound": "hbm", "achieved": k["bytes"] / sec / 1e9, "peak": peaks["hbm_gbs"],
                 "unit": "GB/s", "peak_source": f"{peak_src} copy bandwidth",
                 "work": "N P x 4 bytes of gradient rows written"}
        elif k["flops"] > 0:
            fp64 = args.precision == "fp64"
            r = {"bound": "alu", "achieved": k["flops"] / sec / 1e12,
                 "peak": fp64_nominal if fp64 else fp32_peak, "unit": "TFLOP/s",
                 "peak_source": "FP64 nominal 1.25 TFLOP/s" if fp64 else
                 "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
        else:
            r = {"bound": "latency", "achieved": None, "peak": None, "unit": None,
                 "work": "dependent recurrences on small tridiagonal matrices; no throughput bound"}
        r["traffic"] = None  # DRAM bytes: the ncu summaries under profiles/
        r["frac"] = r["achieved"] / r["peak"] if r.get("peak") and r.get("achieved") else None
        # a persistent grid confined to part of the GPU (the contractions
        # beside the Lanczos kernel): the SMs it had and its fraction of
        # their share of the peak
        sms = k.get("sm_ms", 0.0) / k["ms"] if k["ms"] > 0 else 0.0
        if r["frac"] is not None and 0 < sms < n_sms - 0.5:
            r["sms"] = round(sms, 1)
            r["frac_of_sms"] = r["frac"] * n_sms / sms
        r["kernel_class"] = cls
        r["kernel"] = kernel_of[cls]
        r["launches_per_step"] = k["launches"] / max(args.steps, 1)
        r["ms_per_step"] = k["ms"] / max(args.steps, 1)
        r["step_share"] = r["ms_per_step"] / ms_step
        return r

    rooflines = {c: class_roofline(c) for c in kern}
    rooflines = {c: r for c, r in rooflines.items() if r}
    # the dominant kernel of the step: the kernel function with the largest
    # device time, its classes' launches together (the OPG, Hessian and
    # exact-digit launches are one persistent tensor-core kernel)
    groups = {"umma_gemm_kernel": [c for c in ("syrk", "hcontract", "digits")
                                   if c in rooflines and rooflines[c]["bound"] == "tensor"]}
    for c, r in rooflines.items():
        if r.get("frac") is not None and not any(c in g for g in groups.values()):
            groups[c] = [c]
    groups = {g: cs for g, cs in groups.items() if cs}

    def group_roofline(cs):
        if len(cs) == 1:
            return dict(rooflines[cs[0]])
        ms = sum(kern[c]["ms"] for c in cs)
        sec = ms * 1e-3
        fl = sum(rooflines[c]["achieved"] * 1e12 * kern[c]["ms"] * 1e-3 for c in cs)  # the classes' flops
        sm_ms = sum(kern[c].get("sm_ms", 0.0) for c in cs)
        r = {"bound": "tensor", "achieved": fl / sec / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
             "peak_source": f"{peak_src} bf16 sustained",
             "work": "the classes' tensor flops: " + ", ".join(f"{c} ({rooflines[c]['work']})" for c in cs),
             "traffic": None}
        r["frac"] = r["achieved"] / r["peak"]
        sms = sm_ms / ms if ms > 0 else 0.0
        if 0 < sms < n_sms - 0.5:
            r["sms"] = round(sms, 1)
            r["frac_of_sms"] = r["frac"] * n_sms / sms
        r["kernel_class"] = "+".join(cs)
        r["kernel"] = "umma_gemm_kernel (" + ", ".join(cs) + " launches)"
        r["launches_per_step"] = sum(kern[c]["launches"] for c in cs) / max(args.steps, 1)
        r["ms_per_step"] = ms / max(args.steps, 1)
        r["step_share"] = r["ms_per_step"] / ms_step
        return r

    dom = max(groups, key=lambda g: sum(kern[c]["ms"] for c in groups[g])) if groups else None
    roof = group_roofline(groups[dom]) if dom else None

    serve = precision = None
    if rank == 0 and world == 1 and args.workload == WORKLOAD:
        if not args.no_precision:
            precision = precision_leg(hm, torch, peaks)
        if not args.no_serve:
            serve = serve_leg(args.serve_leg_seconds, args.serve_rate, args.serve_slots, torch)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: MLP {pb.widths} {'/'.join(pb.acts)}, P={P}, "
                                   f"N={N}; " + " + ".join({"opg": "OPG", "hessian": "exact Hessian",
                                                            "eig": f"top-{K_EIG_W} OPG eig"}[c]
                                                           for c in calls) + " per step",
                       "precision": args.precision, "P": P, "N": N, "k": K_EIG_W,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "parallelism": f"replicas x{world}",
                       "step": ("one hess_curvature call (two compute and two copy streams)" if fused else
                                ("single calls on two handles and streams" if two else
                                 "single calls in turn")),
                       **({"only": args.only} if args.only else {})},
            "roofline": roof,
            "rooflines": rooflines,
            "cpu_baseline": ({"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"],
                              "kind": "oracle", "sample": cpu["sample"]}
                             if cpu and "value" in cpu else cpu),
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64_plain": fp64,
            "fp64_probe": probe,
            "serve": serve,
            "precision_opg": precision,
            "kernels_ms_per_step": {k: v["ms"] / max(args.steps, 1) for k, v in kern.items()},
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
