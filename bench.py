"""Benchmark of the sparse GEE hot path on GB300.

One step = one full embedding (all options on) of the workload graph through the C ABI:
label counts and checks, CSR build (radix sort by source), degrees and node table,
label-gather product with the fused epilogue.  Inputs are resident in HBM; L2 is flushed
(256 MiB write) before every timed step, outside the timed interval.

The headline workload is the largest single-graph configuration, the Chung-Lu graph of
600,000 nodes and 10M undirected edges (K = 50).  The timed steps call gee_embed, the
public entry point (from its third call with the same arguments it replays a cached CUDA
graph of its kernels).  Prints ONE JSON line (rank 0):
  roofline      the dominant kernel, from per-kernel CUDA-event times of gee_embed_timed
                calls run right after the timed steps (events between kernels would add
                a few microseconds to every timed step)
  hot_l2        the same call back to back without the flush
  e2e           the same metric through gee_embed_host (pinned host buffers, copies timed)
  cpu_baseline  the FP64 oracle on this host: single thread, and row-parallel on all cores
  configs       (one GPU, default run) the other workloads as sub-records: SBM N=10,000
                (weighted), SBM N=2,000, the 4,096-graph batch (with the one-graph-per-
                launch comparison) and the continuous-batching server (median of repeated
                runs, with their spread)

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload cl600k|sbm10k|sbm2k|batch|serve]
                  [--no-sub] [--no-cpu-baseline]
  python bench.py --impl reference ...     (the oracle arm)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GEE edges/s and % HBM roofline (all options on); p50/p99 served latency"
UNIT = "edges/s"
ALL_OPTIONS = 7
L2_FLUSH_BYTES = 256 << 20
ONE_PASS_BITS = 8  # graphs with node ids of at most this many bits are sorted in one radix pass
KERNEL_TIMING_STEPS = 50
HOT_L2_STEPS = 50              # back-to-back calls without the flush, reported as hot_l2
SUB_STEPS = 100                # timed steps of a single-graph sub-record
SERVE_REPS = 5                 # repeated serving runs (median and spread reported)
CPU_SINGLE_BUDGET_S = 10.0     # bounded CPU-baseline samples
CPU_ALL_BUDGET_S = 5.0

WORKLOADS = {
    "cl600k": dict(desc="Chung-Lu N=600,000, 10M undirected edges (deduplicated, both directions stored), "
                        "gamma 2.1, K=50 Zipf(1.2) classes, unweighted, all options (diag-aug + Laplacian + "
                        "correlation), seed 3"),
    "sbm10k": dict(desc="SBM N=10,000, K=3, priors [0.2,0.3,0.5], p_in 0.13, p_out 0.10 "
                        "(~5.56M undirected edges, both directions stored), fp32 weights U(0,1], "
                        "all options, seed 2"),
    "sbm2k": dict(desc="SBM N=2,000, K=3, priors [0.2,0.3,0.5], p_in 0.13, p_out 0.10, unweighted, "
                       "all options, seed 1"),
    "batch": dict(desc="4,096 graphs in one launch sequence (CUDA graph): N log-uniform [100, 50,000], mean "
                       "degree U[5,200], SBM or Chung-Lu (gamma 2.1) per graph, K U{2..64}, weights U(0,1], "
                       "all options, seed 4"),
    "serve": dict(desc="continuous-batching server: Poisson arrivals of graphs from the batch mix (256 distinct "
                       "graphs) plus 1% large Chung-Lu graphs (N=2M, 100M undirected edges, K=16), pinned host "
                       "inputs, 64 GiB device budget, 2 compute streams, all options, seed 5"),
}


def make_graph(name, rank=0):
    from synth import chung_lu, sbm
    if name == "sbm10k":
        return sbm(10_000, seed=2 + 1000 * rank, weighted=True)
    if name == "sbm2k":
        return sbm(2_000, seed=1 + 1000 * rank)
    if name == "cl600k":
        return chung_lu(600_000, 10_000_000, seed=3 + 1000 * rank)
    raise ValueError(name)


# ---- algorithmic bytes per launch of each kernel ----------------------------------------

def kernel_bytes(g):
    """Algorithmic DRAM bytes of one launch of each kernel: every array the kernel must
    read or write once, nothing for re-reads or L2-resident gathers."""
    E, N, K = g.E, g.N, g.K
    wt = 1 if g.w is not None else 0
    two = max(1, (N - 1).bit_length()) > ONE_PASS_BITS  # the library's kOnePassBits
    b = {}
    b["k_prep"] = 4 * E + 4 * N                                         # src, labels
    if two:
        b["k_scatter_first"] = E * (8 + 4 * wt) + E * (4 + 4 * wt)   # read src/dst/w, write packed/w
        b["k_count"] = 4 * E + 4 * N                                  # read packed, row lengths
        b["k_scatter_final"] = E * (4 + 4 * wt) + E * (4 + 4 * wt)   # read packed/w, write col/val
    else:
        b["k_scatter_final"] = E * (8 + 4 * wt) + E * (4 + 4 * wt)   # read src/dst/w, write col/val
    b["k_rowscan"] = 4 * N + 4 * (N + 1) + (0 if wt else 4 * N + 16 * N)
    b["k_wdeg"] = 4 * E + 4 * (N + 1) + 4 * N + 16 * N if wt else 0
    b["k_spmm"] = E * (4 + 4 * wt) + 4 * (N + 1) + 8 * N + 4 * N + 4 * N * K
    return b


# ---- helpers ----------------------------------------------------------------------------

def reduce_over_ranks(total_ms, edges, device):
    """(max of total_ms, sum of edges) over the ranks of the default process group: the
    job's time is its slowest rank's, its work every rank's graph together."""
    import torch
    import torch.distributed as dist
    m = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    e = torch.tensor([int(edges)], dtype=torch.int64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(m.item()), int(e.item())


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, f in enumerate(fl) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_model():
    """CPU model of this host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
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


def time_oracle(g, threads=None, budget_s=CPU_SINGLE_BUDGET_S, max_calls=1000):
    """Seconds per full-graph oracle call: the plain oracle (threads None) or its row-parallel
    restatement on `threads` host threads (bit-identical results)."""
    import oracle
    call = (lambda: oracle.embed_graph(g, ALL_OPTIONS)) if threads is None else \
        (lambda: oracle.embed_rows_graph(g, ALL_OPTIONS, threads))
    call()  # warm (page-in, build)
    times = []
    t_end = time.perf_counter() + budget_s
    while len(times) < max_calls and (not times or time.perf_counter() < t_end):
        t0 = time.perf_counter()
        call()
        times.append(time.perf_counter() - t0)
    return times


def cpu_baseline(g):
    """The FP64 oracle on this host, single thread and row-parallel on every core."""
    nproc = os.cpu_count() or 1
    t1 = time_oracle(g, None, CPU_SINGLE_BUDGET_S)
    ta = time_oracle(g, nproc, CPU_ALL_BUDGET_S)
    model = cpu_model()
    one = g.E / (sum(t1) / len(t1))
    allc = g.E / (sum(ta) / len(ta))
    return {"value": one, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(t1)} full-graph oracle calls ({g.E} directed edges each), {sum(t1):.1f} s, "
                      "single thread",
            "cpu_model": model, "nproc": nproc,
            "all_cores": {"value": allc, "unit": UNIT, "cores": nproc, "kind": "oracle (row-parallel form, "
                          "bit-identical)", "cpu_model": model,
                          "sample": f"{len(ta)} full-graph calls on {nproc} threads, {sum(ta):.1f} s"}}


# ---- arms -------------------------------------------------------------------------------

def reference_arm(args):
    """The oracle arm: the FP64 oracle on all host cores (its row-parallel form, bit-identical
    to the plain one), one full-graph call per step."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    g = make_graph(args.workload)
    import oracle
    nproc = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.embed_rows_graph(g, ALL_OPTIONS, nproc)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.embed_rows_graph(g, ALL_OPTIONS, nproc)
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    v = g.E / mean
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "N": g.N, "E": g.E, "K": g.K},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nproc, "kind": "oracle (row-parallel form)",
                             "cpu_model": cpu_model(),
                             "sample": f"full graph per step ({g.E} directed edges), {nproc} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batch_kernel_bytes(specs, graphs):
    """Sum over the graphs of kernel_bytes (algorithmic DRAM bytes per kernel launch)."""
    from synth.graphs import Graph
    tot = {}
    for sp, (src, dst, w, y) in zip(specs, graphs):
        stub = Graph(np.empty(0, np.int32), np.empty(0, np.int32), None if w is None else np.empty(0, np.float32),
                     np.empty(0, np.int32), sp["N"], sp["K"])
        stub.src = np.broadcast_to(np.int32(0), (sp["E"],))
        for k, v in kernel_bytes(stub).items():
            tot[k] = tot.get(k, 0) + v
    return tot


def measure_batch(gee, dev, n_graphs, steps, warmup, rank=0):
    """The many-graph batch: `steps` CUDA-event-timed replays of one plan (CUDA graph) with
    the automatic tuning fields, then with the fields of the batch tuner; the per-kernel
    roofline of one extra timed launch; and the plain one-graph-per-launch path over the
    same graphs on the same stream.  Frees its device memory before returning."""
    import torch
    from synth import batch_specs
    from synth.torch_batch import batch_graph_torch
    specs = batch_specs(n_graphs, seed=4 + 1000 * rank)
    graphs = [batch_graph_torch(sp, dev) for sp in specs]
    torch.cuda.synchronize()
    E_tot = sum(sp["E"] for sp in specs)
    items = [(s, d, w, y, sp["N"], sp["K"]) for (s, d, w, y), sp in zip(graphs, specs)]
    stream = torch.cuda.current_stream(dev)
    names = gee.PHASES

    def run(opts):
        plan = gee.BatchPlan(items, opts=opts)
        for _ in range(max(warmup, 3)):
            plan.launch(stream, use_graph=True)
        torch.cuda.synchronize()
        if int(plan.status.abs().sum().item()) != 0:
            raise RuntimeError("device status set")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for i in range(steps):
            ev[i][0].record(stream)
            plan.launch(stream, use_graph=True, status=False)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        # per-kernel times of one extra (timed) launch of the same plan
        phase = np.zeros(gee_phase_count(), np.float32)
        plan.launch_timed(phase, stream)
        plan.close()
        del plan
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return ms, phase

    heur_ms, _ = run(gee.make_opts(ALL_OPTIONS))
    # the batch tuner (outside the timed region; it times whole launches itself)
    best, tune_ms = gee.batch_autotune(items, ALL_OPTIONS, stream)
    torch.cuda.empty_cache()
    ms_per_step, phase = run(best)
    kb = batch_kernel_bytes(specs, graphs)
    kernels = {names[i]: float(phase[i]) for i in range(len(names))
               if phase[i] > 0 and names[i] in kb and kb[names[i]] > 0}
    dom = max(kernels, key=lambda k: kernels[k])
    peaks = load_peaks()
    per_kernel = {k: {"ms": round(v, 4), "alg_bytes": int(kb[k]), "gbs": round(kb[k] / (v * 1e-3) / 1e9, 1),
                      "frac": round(kb[k] / (v * 1e-3) / 1e9 / peaks["hbm_gbs"], 3)} for k, v in kernels.items()}
    achieved = kb[dom] / (kernels[dom] * 1e-3) / 1e9
    # the plain one-graph-per-launch path over the same graphs, same stream, same accuracy
    opts = gee.make_opts(ALL_OPTIONS)
    wsz = max(gee.gee_workspace_size(sp["E"], sp["N"], sp["K"], True, opts) for sp in specs)
    wsb = torch.empty(wsz, dtype=torch.uint8, device=dev)
    Zs = [torch.empty((sp["N"], sp["K"]), dtype=torch.float32, device=dev) for sp in specs]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(2):
        a.record(stream)
        for (s_, d_, w_, y_), sp, Z in zip(graphs, specs, Zs):
            rc = gee.gee_embed(s_, d_, w_, sp["E"], sp["N"], y_, sp["K"], opts, Z, wsb, wsz, stream, None)
            if rc:
                raise RuntimeError(gee.gee_strerror(rc))
        b.record(stream)
        torch.cuda.synchronize()
    solo_ms = a.elapsed_time(b)
    launches = int(sum(1 for i, n in enumerate(names) if phase[i] >= 0 and n != "memset"))
    out = {"value": E_tot / (ms_per_step * 1e-3), "unit": UNIT, "ms_per_step": ms_per_step, "steps": steps,
           "workload": WORKLOADS["batch"]["desc"], "graphs": len(specs), "E": E_tot,
           "N": sum(sp["N"] for sp in specs), "l2": "inputs (~40 GB) far larger than L2",
           "tuning": {"source": "gee_batch_autotune", "vec_width": int(best.vec_width),
                      "short_len": int(best.short_len), "rows_per_item": int(best.rows_per_item),
                      "autotune_ms_per_launch": round(tune_ms, 3)},
           "heuristic": {"ms_per_step": heur_ms, "value": E_tot / (heur_ms * 1e-3), "unit": UNIT,
                         "note": "the same plan with the automatic tuning fields"},
           "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                        "peak_source": peaks["source"], "traffic": traffic_for(dom, "batch"),
                        "alg_bytes_per_launch": int(kb[dom]), "kernels": per_kernel},
           "one_graph_per_launch": {"value": E_tot / (solo_ms * 1e-3), "unit": UNIT, "ms": solo_ms},
           "gpu_launches_per_step": launches}
    del graphs, wsb, Zs, items
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def batch_arm(args, ws_n, rank, local, dev):
    import torch
    import paper_2406_03726_gb300 as gee
    if ws_n > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        m = measure_batch(gee, dev, args.batch_graphs, args.steps, args.warmup, rank)
    total_ms = m["ms_per_step"] * args.steps
    E_job = m["E"]
    if ws_n > 1:
        total_ms, E_job = reduce_over_ranks(total_ms, m["E"], dev)
    ms_per_step = total_ms / args.steps
    line = {"metric": METRIC, "value": E_job / (ms_per_step * 1e-3), "unit": UNIT, "n_gpus": ws_n,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": m["workload"], "graphs": m["graphs"], "E": m["E"], "N": m["N"], "l2": m["l2"],
                       "parallelism": f"replicas x{ws_n} (independent batches, no collective)"},
            "roofline": m["roofline"], "one_graph_per_launch": m["one_graph_per_launch"],
            "tuning": m["tuning"], "heuristic": m["heuristic"],
            "e2e": None, "e2e_note": "not measured for the batch (about 40 GB of host input)",
            "gpu_launches": m["gpu_launches_per_step"] * args.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line))
    return 0


def _serve_once(gee, reqs, gaps):
    """One serving run: requests `reqs` submitted at once (gaps None) or with the given
    inter-arrival gaps in seconds; each request's latency runs from its submission to its
    Z being ready."""
    import threading
    srv = gee.Server(64 << 30, ALL_OPTIONS, max_batch=1024, streams=2)
    tickets = [None] * len(reqs)

    def submitter():
        t_next = time.perf_counter()
        for i, ((s_, d_, w_, y_), sp) in enumerate(reqs):
            if gaps is not None:
                t_next += gaps[i]
                while True:
                    dt = t_next - time.perf_counter()
                    if dt <= 0:
                        break
                    time.sleep(min(dt, 0.002))
            tickets[i] = srv.submit(s_.numpy(), d_.numpy(), w_.numpy(), y_.numpy(), sp["N"], sp["K"])

    th = threading.Thread(target=submitter)
    t_start = time.perf_counter()
    th.start()
    lat = []
    t_last = t_start
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0001)
        res = srv.poll(tickets[i], wait=True)
        if res is None:
            raise RuntimeError("request did not complete")
        lat.append(res[2])
        t_last = time.perf_counter()
        srv.release(tickets[i])
    th.join()
    st = srv.stats()
    srv.close()
    edges = sum(sp["E"] for _, sp in reqs)
    span = t_last - t_start
    lat = np.array(lat)
    return {"requests": len(reqs), "edges": int(edges), "seconds": span, "edges_per_s": edges / span,
            "req_per_s": len(reqs) / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "launches": int(st["launches"]),
            "peak_pool_bytes": int(st["peak_bytes_in_use"]), "pool_bytes": int(st["pool_bytes"])}


def _median_spread(runs, keys=("edges_per_s", "p50_ms", "p99_ms", "req_per_s")):
    out = {}
    for k in keys:
        v = [r[k] for r in runs]
        out[k] = statistics.median(v)
        out[k + "_min"] = min(v)
        out[k + "_max"] = max(v)
    out["runs"] = len(runs)
    out["requests_per_run"] = runs[0]["requests"]
    return out


def measure_serving(gee, dev, R, reps, rank=0):
    """The continuous-batching server: `reps` repetitions of (saturation, 50% and 90% of
    that repetition's saturation rate), each of R requests; medians with min and max."""
    import torch
    from synth import batch_specs
    from synth.torch_batch import batch_graph_torch
    rng = np.random.default_rng(5 + 1000 * rank)
    specs = batch_specs(256, seed=5 + 1000 * rank)
    big = {"index": -1, "N": 2_000_000, "m": 100_000_000, "E": 200_000_000, "K": 16, "kind": "chung_lu",
           "seed": 77 + rank}

    def to_host(sp):
        src, dst, w, y = batch_graph_torch(sp, dev)
        pin = [t.cpu().pin_memory() for t in (src, dst, w, y)]
        del src, dst, w, y
        return pin, sp

    pool = [to_host(sp) for sp in specs]
    big_host = to_host(big)
    torch.cuda.empty_cache()

    def draw(n):
        return [big_host if rng.random() < 0.01 else pool[rng.integers(len(pool))] for _ in range(n)]

    # one seeded trace per load level, replayed by every repetition: the spread over the
    # repetitions is the system's, not the draw's
    trace = draw(R)
    unit_gaps = rng.exponential(1.0, R)           # Poisson arrivals at rate 1, scaled below
    _serve_once(gee, draw(50), None)              # warm-up
    sat = [_serve_once(gee, trace, None) for _ in range(reps)]
    rate = statistics.median(r["req_per_s"] for r in sat)
    r50 = [_serve_once(gee, trace, unit_gaps / (0.5 * rate)) for _ in range(reps)]
    r90 = [_serve_once(gee, trace, unit_gaps / (0.9 * rate)) for _ in range(reps)]
    torch.cuda.empty_cache()
    return {"workload": WORKLOADS["serve"]["desc"], "saturation": _median_spread(sat),
            "at_50pct": _median_spread(r50), "at_90pct": _median_spread(r90),
            "trace": {"requests": R, "large_graphs": sum(1 for _, sp in trace if sp["N"] == big["N"]),
                      "edges": int(sum(sp["E"] for _, sp in trace))},
            "note": "median over repeated runs of one seeded trace, with min and max; the 50% and 90% "
                    "arrival rates are fractions of the median saturation rate",
            "h2d_bytes_per_request": int(sum(sp["E"] * 12 + sp["N"] * 4 for _, sp in trace) / R)}


def serve_arm(args, ws_n, rank, local, dev):
    import paper_2406_03726_gb300 as gee
    R = max(200, args.steps)
    with ClockSampler(local) as clk:
        m = measure_serving(gee, dev, R, SERVE_REPS, rank)
    sat = m["saturation"]
    line = {"metric": METRIC, "value": sat["edges_per_s"] * ws_n, "unit": UNIT, "n_gpus": ws_n, "steps": R,
            "warmup": 50, "ms_per_step": 1e3 / sat["req_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": m["workload"], "requests_per_run": R,
                       "parallelism": f"replicas x{ws_n} (independent servers, no collective)"},
            "serving": m,
            "e2e": {"value": sat["edges_per_s"], "unit": UNIT, "h2d_bytes_per_step": m["h2d_bytes_per_request"],
                    "d2h_bytes_per_step": 0,
                    "note": "host inputs in, Z resident on the device (the serving contract)"},
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line))
    return 0


def measure_single(gee, g, dev, steps, warmup, workload, barrier=None, fixed=None):
    """One graph: autotuned options, `steps` L2-flushed CUDA-event-timed gee_embed calls,
    per-kernel times of gee_embed_timed calls right after, hot-L2 calls and the end-to-end
    host-buffer path.  Returns the record (no cross-rank reduction)."""
    import torch
    E, N, K = g.E, g.N, g.K
    t = lambda a: None if a is None else torch.from_numpy(a).to(dev)
    src, dst, w, y = t(g.src), t(g.dst), t(g.w), t(g.labels)
    # the project's autotuner picks the tuning fields for this graph (outside the timed
    # region; it times candidate calls itself), unless they are given (profiling runs)
    if fixed is None:
        opts, tune_ms = gee.autotune(src, dst, w, N, y, K, ALL_OPTIONS)
    else:
        opts, tune_ms = gee.make_opts(ALL_OPTIONS, fixed[0], 0, fixed[1], fixed[2], fixed[3]), 0.0
    tuned = {"hub_threshold": int(opts.hub_threshold), "rows_per_item": int(opts.rows_per_item),
             "autotune_ms_per_call": round(tune_ms, 4), "source": "autotune" if fixed is None else "--opts"}
    for f in ("vec_width", "short_len"):
        if hasattr(opts, f):
            tuned[f] = int(getattr(opts, f))
    nbytes = gee.gee_workspace_size(E, N, K, w is not None, opts)
    wsb = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    Z = torch.empty((N, K), dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    phase = np.zeros(gee_phase_count(), np.float32)

    def step_plain():
        rc = gee.gee_embed(src, dst, w, E, N, y, K, opts, Z, wsb, nbytes, stream, status)
        if rc:
            raise RuntimeError(gee.gee_strerror(rc))

    for _ in range(max(warmup, 3)):
        step_plain()
        # the timed call is the one the timed region repeats: its first call launches
        # directly, the second captures its launch graph, later ones replay it
        rc = gee.gee_embed_timed(src, dst, w, E, N, y, K, opts, Z, wsb, nbytes, stream, status, phase)
        if rc:
            raise RuntimeError(gee.gee_strerror(rc))
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())}")

    # ---- timed region: `steps` calls of the public entry point, each bracketed by CUDA
    # events on the launch stream (from the third call on, gee_embed replays its graph)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    n_kt = min(steps, KERNEL_TIMING_STEPS)
    phase_sum = np.zeros_like(phase)
    phase_cnt = np.zeros_like(phase)
    if barrier:
        barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))               # L2 flush, outside the timed interval
        ev[i][0].record(stream)
        step_plain()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    # ---- kernel timing, right after: the same call with CUDA events between its kernels
    # (gee_embed_timed), which the timed steps leave out because each event pair adds a
    # few microseconds to the step
    for i in range(n_kt):
        flush.fill_(float(i))
        rc = gee.gee_embed_timed(src, dst, w, E, N, y, K, opts, Z, wsb, nbytes, stream, status, phase)
        if rc:
            raise RuntimeError(gee.gee_strerror(rc))
        ok = phase >= 0
        phase_sum[ok] += phase[ok]
        phase_cnt[ok] += 1
    torch.cuda.synchronize()
    # ---- hot-L2 steps: the same call without the flush, so a graph whose arrays fit in
    # L2 is served from it (reported beside the flushed number, not as the value)
    n_hot = min(steps, HOT_L2_STEPS)
    ev_hot = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_hot)]
    step_plain()
    for i in range(n_hot):
        ev_hot[i][0].record(stream)
        step_plain()
        ev_hot[i][1].record(stream)
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())}")
    # ---- re-embedding with new labels on the CSR the last call built (gee_reembed), the
    # iterative / predicted-labels use: L2-flushed calls with a permutation of the labels
    gen = torch.Generator(device=dev)
    gen.manual_seed(9)
    y2 = y[torch.randperm(N, generator=gen, device=dev)].contiguous()
    Z2 = torch.empty_like(Z)
    for _ in range(3):  # seen, captured, replayed
        rc = gee.gee_reembed(y2, E, N, K, w is not None, opts, Z2, wsb, nbytes, stream, status)
        if rc:
            raise RuntimeError(gee.gee_strerror(rc))
    n_re = min(steps, KERNEL_TIMING_STEPS)
    ev_re = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_re)]
    for i in range(n_re):
        flush.fill_(float(i))
        ev_re[i][0].record(stream)
        gee.gee_reembed(y2, E, N, K, w is not None, opts, Z2, wsb, nbytes, stream, status)
        ev_re[i][1].record(stream)
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())} after gee_reembed")
    re_ms = float(np.mean([a.elapsed_time(b) for a, b in ev_re]))
    step_ms = [a.elapsed_time(b) for a, b in ev]
    hot_ms = float(np.median([a.elapsed_time(b) for a, b in ev_hot])) if n_hot else None
    total_ms = sum(step_ms)
    ms_per_step = total_ms / steps

    # ---- per-kernel roofline of the dominant kernel
    names = gee.PHASES
    avg = {names[i]: float(phase_sum[i] / phase_cnt[i]) for i in range(len(names)) if phase_cnt[i] > 0}
    kb = kernel_bytes(g)
    kernels = {k: v for k, v in avg.items() if k in kb and kb[k] > 0}
    dom = max(kernels, key=lambda k: kernels[k])
    peaks = load_peaks()
    achieved = kb[dom] / (kernels[dom] * 1e-3) / 1e9
    per_kernel = {k: {"ms": round(float(v), 5), "alg_bytes": int(kb[k]),
                      "gbs": round(kb[k] / (v * 1e-3) / 1e9, 1),
                      "frac": round(kb[k] / (v * 1e-3) / 1e9 / peaks["hbm_gbs"], 3)}
                  for k, v in kernels.items()}
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "peak_source": peaks["source"], "traffic": traffic_for(dom, workload),
                "alg_bytes_per_launch": int(kb[dom]), "kernels": per_kernel,
                "kernel_timing": f"CUDA events between the kernels of gee_embed_timed, {n_kt} L2-flushed "
                                 "calls right after the timed steps, same process and clock sampling"}
    # the whole step against the end-to-end algorithmic bytes (COO read once, CSR written
    # once, then the product's bytes)
    b_e2e = e2e_alg_bytes(g)
    roofline["step"] = {"alg_bytes": int(b_e2e), "gbs": round(b_e2e / (ms_per_step * 1e-3) / 1e9, 1),
                        "frac": round(b_e2e / (ms_per_step * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}

    # ---- end to end through the host-buffer entry point (pinned memory)
    e2e = e2e_measure(gee, g, dev, stream, opts, steps)
    launches = int(sum(1 for i, n in enumerate(names) if phase_cnt[i] > 0 and n != "memset"))  # per step
    out = {"value": E / (ms_per_step * 1e-3), "unit": UNIT, "ms_per_step": ms_per_step, "steps": steps,
           "opts": opts, "total_ms": total_ms, "workload": WORKLOADS[workload]["desc"], "N": N, "E": E, "K": K,
           "tuning": tuned, "roofline": roofline, "e2e": e2e, "gpu_launches_per_step": launches,
           "l2": "flushed before every step (256 MiB write, untimed)"}
    if hot_ms is not None:
        out["hot_l2"] = {"ms_per_step": round(hot_ms, 5), "value": E / (hot_ms * 1e-3), "unit": UNIT,
                         "steps": n_hot, "note": "median of back-to-back calls without the L2 flush"}
    out["reembed"] = {"ms_per_call": round(re_ms, 5), "value": E / (re_ms * 1e-3), "unit": UNIT, "calls": n_re,
                      "speedup_vs_embed": round(ms_per_step / re_ms, 2),
                      "note": "gee_reembed with permuted labels on the CSR, degrees and plans of the last call "
                              "(L2 flushed before each call)"}
    del src, dst, w, y, y2, wsb, Z, Z2, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def measure_symmetrize(gee, g, dev, steps, opts):
    """The same graph given once per undirected edge (the entries with source < target)
    with GEE_SYMMETRIZE: the CSR build makes the reverse copies.  L2-flushed CUDA-event
    steps, kernel times from gee_embed_timed, and the host-buffer path (half the input)."""
    import torch
    from synth.graphs import Graph
    one = g.src < g.dst
    h = Graph(g.src[one], g.dst[one], None if g.w is None else g.w[one], g.labels, g.N, g.K)
    E_in, N, K = h.E, h.N, h.K
    o = gee.make_opts(ALL_OPTIONS | gee.SYMMETRIZE, opts.hub_threshold, opts.lanes_per_row, opts.rows_per_item,
                      opts.vec_width, opts.short_len)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    src, dst, w, y = t(h.src), t(h.dst), t(h.w), t(h.labels)
    nbytes = gee.gee_workspace_size(E_in, N, K, w is not None, o)
    wsb = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    Z = torch.empty((N, K), dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    phase = np.zeros(gee_phase_count(), np.float32)
    for _ in range(3):
        gee.gee_embed(src, dst, w, E_in, N, y, K, o, Z, wsb, nbytes, stream, status)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        rc = gee.gee_embed(src, dst, w, E_in, N, y, K, o, Z, wsb, nbytes, stream, status)
        ev[i][1].record(stream)
        if rc:
            raise RuntimeError(gee.gee_strerror(rc))
    torch.cuda.synchronize()
    acc, cnt = np.zeros_like(phase), np.zeros_like(phase)
    for i in range(min(steps, KERNEL_TIMING_STEPS)):
        flush.fill_(float(i))
        gee.gee_embed_timed(src, dst, w, E_in, N, y, K, o, Z, wsb, nbytes, stream, status, phase)
        acc[phase >= 0] += phase[phase >= 0]
        cnt[phase >= 0] += 1
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())} with GEE_SYMMETRIZE")
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    names = gee.PHASES
    kern = {names[i]: round(float(acc[i] / cnt[i]), 5) for i in range(len(names))
            if cnt[i] > 0 and names[i] != "memset" and acc[i] > 0}
    E_csr = g.E  # entries of A: both directions of every undirected edge (no self-loops here)
    wt = 1 if h.w is not None else 0
    first = E_in * (8 + 4 * wt) + E_csr * (4 + 4 * wt)  # input read once, both copies written
    peaks = load_peaks()
    e2e = e2e_measure(gee, h, dev, stream, o, steps)
    e2e["value"] = E_csr * e2e["value"] / E_in       # the metric counts entries of A
    del src, dst, w, y, wsb, Z, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return {"ms_per_step": round(ms, 5), "value": E_csr / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "input_edges": E_in, "csr_entries": E_csr, "kernels_ms": kern,
            "k_scatter_first": {"alg_bytes": int(first), "frac": round(first / (kern["k_scatter_first"] * 1e-3) / 1e9 /
                                                                      peaks["hbm_gbs"], 4)},
            "e2e": e2e,
            "note": "the graph given once per undirected edge with GEE_SYMMETRIZE (same tuning fields); "
                    "value counts the entries of A; the first radix pass reads the input once for both "
                    "directions"}


def measure_sparse(gee, g, dev, steps, K):
    """Sparse Z (gee_embed_sparse) of the graph with its labels redrawn from K classes
    (every fifth node unlabelled, seed 137): L2-flushed CUDA-event-timed calls."""
    import torch
    rng = np.random.default_rng(137)
    y_np = rng.integers(0, K, g.N).astype(np.int32)
    y_np[::5] = -1
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    src, dst, w, y = t(g.src), t(g.dst), t(g.w), t(y_np)
    o = gee.make_opts(ALL_OPTIONS)
    n = gee.gee_sparse_workspace_size(g.E, g.N, K, w is not None, o)
    ws = torch.empty(n, dtype=torch.uint8, device=dev)
    cap = g.E + g.N
    zr = torch.empty(g.N + 1, dtype=torch.int32, device=dev)
    zc = torch.empty(cap, dtype=torch.int32, device=dev)
    zv = torch.empty(cap, dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def call():
        rc = gee.gee_embed_sparse(src, dst, w, g.E, g.N, y, K, o, zr, zc, zv, cap, ws, n, stream, status)
        if rc:
            raise RuntimeError(gee.gee_strerror(rc))

    for _ in range(3):
        call()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        call()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())} in gee_embed_sparse")
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    nnz = int(zr[g.N].item())
    del src, dst, w, y, ws, zr, zc, zv, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return {"K": K, "ms_per_call": round(ms, 4), "value": g.E / (ms * 1e-3), "unit": UNIT, "nnz": nnz,
            "dense_z_bytes": 4 * g.N * K, "sparse_z_bytes": 8 * nnz + 4 * (g.N + 1), "calls": steps,
            "note": "gee_embed_sparse: CSR build, then Z as CSR over classes (labels redrawn from K classes, "
                    "every fifth node unlabelled); L2 flushed before each call"}


def e2e_alg_bytes(g):
    """Algorithmic bytes of a whole step from the edge list: the COO read once, the CSR
    written once, and the product's bytes."""
    wt = 1 if g.w is not None else 0
    return g.E * (8 + 4 * wt) + g.E * (4 + 4 * wt) + kernel_bytes(g)["k_spmm"]


def gpu_arm(args):
    import torch
    import paper_2406_03726_gb300 as gee

    ws_n, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws_n > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.workload in ("batch", "serve"):
        rc = (batch_arm if args.workload == "batch" else serve_arm)(args, ws_n, rank, local, dev)
        if ws_n > 1:
            torch.distributed.destroy_process_group()
        return rc
    g = make_graph(args.workload, rank)
    barrier = torch.distributed.barrier if ws_n > 1 else None
    subs = {}
    with ClockSampler(local) as clk:
        fixed = tuple(int(x) for x in args.opts.split(",")) if args.opts else None
        m = measure_single(gee, g, dev, args.steps, args.warmup, args.workload, barrier, fixed)
        # the other workloads as sub-records (one GPU, default run)
        if ws_n == 1 and not args.no_sub:
            for name in ("sbm10k", "sbm2k"):
                if name != args.workload:
                    subs[name] = measure_single(gee, make_graph(name), dev, min(args.steps, SUB_STEPS),
                                                args.warmup, name)
                    subs[name].pop("opts")
            subs["batch"] = measure_batch(gee, dev, args.batch_graphs, 3, 3)
            subs["serving"] = measure_serving(gee, dev, 200, SERVE_REPS)
    total_ms, E_job = m["total_ms"], g.E
    if ws_n > 1:
        total_ms, E_job = reduce_over_ranks(total_ms, g.E, dev)
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = E_job / (ms_per_step * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": m["workload"], "name": args.workload, "N": g.N, "E": g.E, "K": g.K,
                       "tuning": m["tuning"], "l2": m["l2"],
                       "parallelism": f"replicas x{ws_n} (independent graphs, no collective)"},
            "roofline": m["roofline"], "e2e": m["e2e"], "gpu_launches": m["gpu_launches_per_step"] * args.steps,
            "clocks": clk.summary()}
    if "hot_l2" in m:
        line["hot_l2"] = m["hot_l2"]
    line["reembed"] = m["reembed"]
    if ws_n == 1 and not args.no_sub and args.workload == "cl600k":
        line["symmetrize"] = measure_symmetrize(gee, g, dev, min(args.steps, SUB_STEPS), m.pop("opts"))
        line["sparse"] = [measure_sparse(gee, g, dev, 20, K) for K in (g.K, 100_000)]
    m.pop("opts", None)
    if subs:
        line["configs"] = subs
    if rank == 0:
        if ws_n == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g)
        print(json.dumps(line))
    if ws_n > 1:
        torch.distributed.destroy_process_group()
    return 0


def sparse_only(args):
    """The sparse-Z record of one workload (one GPU), as one JSON line."""
    import torch
    import paper_2406_03726_gb300 as gee
    dev = torch.device("cuda", 0)
    g = make_graph(args.workload)
    rec = measure_sparse(gee, g, dev, args.steps, args.sparse_k)
    print(json.dumps({"workload": WORKLOADS[args.workload]["desc"], "sparse": rec}))
    return 0


def gee_phase_count():
    return 16  # room for the GEE_NUM_PHASES floats gee_embed_timed writes


def e2e_measure(gee, g, dev, stream, opts, steps):
    import torch
    E, N, K = g.E, g.N, g.K
    n = gee.gee_host_workspace_size(E, N, K, g.w is not None, opts)
    wsb = torch.empty(n, dtype=torch.uint8, device=dev)
    pin = lambda a: None if a is None else torch.from_numpy(a).pin_memory()
    src, dst, w, y = pin(g.src), pin(g.dst), pin(g.w), pin(g.labels)
    Z = torch.empty((N, K), dtype=torch.float32).pin_memory()
    st = np.zeros(1, np.uint32)

    def call():
        rc = gee.gee_embed_host(src, dst, w, E, N, y, K, opts, Z, wsb, n, stream, st)
        if rc:
            raise RuntimeError(gee.gee_strerror(rc))

    for _ in range(3):
        call()
    steps = max(3, min(steps, 100))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        call()                      # synchronous: returns with Z in host memory
    dt = (time.perf_counter() - t0) / steps
    h2d = 8 * E + (4 * E if g.w is not None else 0) + 4 * N
    d2h = 4 * N * K + 4
    return {"value": E / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "host_memory": "pinned"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s"}


def traffic_for(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary (profiles/traffic.json),
    or None when there is none or it was taken on a different kernel source."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2406_03726_gb300", "csrc", "gee_kernels.cu")
    try:
        d = json.load(open(p))
        if d.get("source_sha1") != hashlib.sha1(open(src, "rb").read()).hexdigest():
            return None
        return d.get(workload, {}).get(kernel)
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gee", choices=["gee", "reference"])
    ap.add_argument("--workload", default="cl600k", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the sub-records of the other workloads")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--sparse-k", type=int, default=0,
                    help="only the sparse-Z measurement of the workload, with labels drawn from this many "
                         "classes (profiling runs)")
    ap.add_argument("--opts", default="", help="hub_threshold,rows_per_item,vec_width,short_len for the main "
                                                "workload instead of the autotuner (profiling runs)")
    args = ap.parse_args()
    if args.sparse_k:
        return sparse_only(args)
    if args.impl == "reference":
        if args.workload in ("batch", "serve"):
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single graphs only"}))
            return 0
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
