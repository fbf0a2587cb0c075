"""Benchmark: temporal motif mining on one GB300 (or N replicas under torchrun).

Default workload (one "step"): the 10M-edge power-law temporal graph (1M
nodes, Zipf 2.1, bursty 3-year timestamps, 10% reciprocated edges), resident in
HBM; each of its four queries (3-cycle, 4-cycle, 3-edge out-star, 4-edge
ping-pong; delta = 3600 s) is counted exactly and enumerated into a
2^26-row buffer by one tm_enumerate call (its count pass gives the total, its
fill pass the rows).  value = root-edges/s = 4 queries x m roots / step time.
Extra objects on the same line: matches/s, the batched form (the 64-query mix
in one CUDA-graph launch vs one query at a time), the served form (Poisson
arrivals, p50/p99 vs serial single-query execution), the hub-skewed graph, the
roofline of the dominant kernel and the CPU oracle baseline.

--impl reference times the CPU oracle itself (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CAP = 1 << 26
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "source": "fallback"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tm", choices=["tm", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="graph size multiplier (1.0 = full workload)")
    ap.add_argument("--no-extras", action="store_true", help="skip batched / served / cpu legs")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--workload", default="powerlaw_10m",
                    choices=["powerlaw_10m", "hubskew_100m", "serve_1b", "count_1b", "batch64", "sweeps"],
                    help="powerlaw_10m: count + enumerate of 4 queries (default); hubskew_100m: count of the "
                         "labelled 5-edge path and the chorded 4-cycle; serve_1b: served Poisson traces on the "
                         "1B-edge graph; count_1b: GPU ingest and counts of the four queries (delta 600 s) "
                         "on the 1B-edge graph; sweeps: constraint sweep (4-cycle N / V / V+T / V+T+A) and the "
                         "ablation over delta on the 10M-edge graph")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return dict(PEAKS_FALLBACK)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_samples(self, n, limit_s=5.0):
        """Block until n samples have arrived (bounded), so the record brackets the timed region."""
        t0 = time.time()
        while self.proc is not None and len(self.lines) < n and time.time() - t0 < limit_s:
            time.sleep(0.01)
        return len(self.lines)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.wait_samples(len(self.lines) + 1, 1.0)    # one sample taken after the timed region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "tm" else "gloo"
        dist.init_process_group(backend)
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(scale, name="powerlaw_10m"):
    import synth
    if name == "hubskew_100m":
        return synth.hub_skewed_100m(scale=scale), synth.hub_skewed_queries()
    if name == "serve_1b":
        return synth.powerlaw_1b(scale=scale), synth.powerlaw_queries(3600)
    g = synth.powerlaw_10m(scale=scale)
    return g, synth.powerlaw_queries(3600)


# --------------------------------------------------------------- CPU oracle

def step_config(g, queries, count_only, ws):
    """The `config` object of both arms' lines (the workload one step covers)."""
    return {"workload": g.name, "n_nodes": g.n_nodes, "n_edges": g.n_edges,
            "queries": [q.name for q in queries], "delta_s": queries[0].delta,
            "enumerate_cap": None if count_only else CAP,
            "step": "count of each query" if count_only else "count + capped enumerate of each query",
            "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{ws}"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(og, queries, m, roots, threads, count_only):
    """One bounded sample of the step: for each query, the roots of a contiguous range of
    `roots` edges (placed at a different offset per query) are counted and, unless
    count_only, enumerated (rows of the range's matches), split into `threads` root
    sub-ranges run at once.  The oracle's library call releases the GIL, so threads run on
    separate cores.  Returns (seconds, root edges covered)."""
    from concurrent.futures import ThreadPoolExecutor
    jobs = []
    for qi, q in enumerate(queries):
        a = (m // (len(queries) + 1)) * (qi + 1)
        a = max(0, min(a, m - roots))
        b = min(m, a + roots)
        cuts = [a + (b - a) * j // threads for j in range(threads + 1)]
        jobs += [(q, x, y) for x, y in zip(cuts[:-1], cuts[1:]) if y > x]

    def run(job):
        q, x, y = job
        c = og.count(q, x, y)
        if not count_only and c:
            og.enumerate(q, cap=min(c, CAP), root_begin=x, root_end=y)
        return y - x

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        done = sum(ex.map(run, jobs))
    return time.perf_counter() - t0, done


def oracle_rate(g, queries, seconds, threads, count_only, og=None):
    """Grow the sample until it takes about `seconds`; returns (root-edges/s, s, roots)."""
    import oracle
    og = og or oracle.Graph.from_synth(g)
    m = g.n_edges
    roots = 1024 * threads
    while True:
        dt, done = oracle_sample(og, queries, m, roots, threads, count_only)
        if dt >= seconds * 0.5 or roots >= m:
            return done / dt, dt, done
        roots = min(m, int(roots * min(16.0, max(2.0, seconds / max(dt, 1e-3)))))


def run_reference(args, rank, ws):
    if rank != 0:
        return
    g, queries = workload(args.scale, args.workload)
    count_only = args.workload == "hubskew_100m"
    import oracle
    t0 = time.perf_counter()
    og = oracle.Graph.from_synth(g)
    build_s = time.perf_counter() - t0
    threads = host_cores()
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    # size one step's sample once (untimed), then time the steps on that sample
    _, _, roots = oracle_rate(g, queries, per_step, threads, count_only, og)
    per_query = max(1, roots // len(queries))
    times, roots_total = [], 0
    for s in range(args.warmup + args.steps):
        dt, done = oracle_sample(og, queries, g.n_edges, per_query, threads, count_only)
        if s >= args.warmup:
            times.append(dt)
            roots_total += done
    value = roots_total / sum(times)
    line = {"impl": "reference", "metric": "root-edges/s", "value": value, "unit": "root-edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": step_config(g, queries, count_only, ws),
            "cpu_baseline": {"value": value, "unit": "root-edges/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step: {per_query} contiguous root edges per query, "
                                       f"{'counted' if count_only else 'counted and enumerated'}, split "
                                       f"into {threads} root ranges on {threads} threads; oracle graph "
                                       f"build {build_s:.1f} s not timed"},
            "e2e": {"value": value, "unit": "root-edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU legs

TRAFFIC_FILE = os.path.join(ROOT, "profiles", "search_count_traffic_powerlaw_10m.json")
KERNEL_SOURCES = ("paper_2310_02800_gb300/csrc/search.cu", "paper_2310_02800_gb300/csrc/tm_internal.cuh",
                  "paper_2310_02800_gb300/csrc/graph.cu")


def kernel_source_hash():
    """Hash of the kernel sources' code: line comments, surrounding blanks and empty
    lines are left out, so an edit to comments alone keeps a capture valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            for line in fh:
                code = re.sub(r"//.*$", "", line).strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def measured_traffic(workload):
    """DRAM bytes of one step's count pass (all its count launches) from the committed ncu
    capture of this kernel on this workload; None when the kernel sources changed since it
    was taken."""
    if workload != "powerlaw_10m" or not os.path.exists(TRAFFIC_FILE):
        return None
    d = json.load(open(TRAFFIC_FILE))
    if d.get("kernel_source_sha256") != kernel_source_hash() or "dram_bytes_count_pass_per_step" not in d:
        return None
    return float(d["dram_bytes_count_pass_per_step"])


def alg_bytes(w, k, matches_written, with_labels=False):
    """Algorithmic bytes of one search: 16 B per root edge (17 with the label column), a
    32 B offset sector per located window, 16 B per window entry plus one per window (the
    read that ends it), 32 B per binary-search probe sector, 4k B per written match row.
    Returns (with probe sectors, without)."""
    root_b = (17 if with_labels else 16) * w["roots"]
    nodes = sum(w["nodes"])
    entries = sum(w["entries"])
    lower = root_b + 32 * nodes + 16 * (entries + nodes) + 4 * k * matches_written
    return lower + 32 * w["probe_sectors"], lower


def main():
    args = parse()
    rank, ws = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, ws)
        return
    import torch
    import synth
    import paper_2310_02800_gb300 as tmg
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    if args.workload == "count_1b":
        return count_1b(args, dev, stream)
    if args.workload == "serve_1b":
        return serve_1b(args, dev)
    if args.workload == "sweeps":
        return sweeps(args, dev, stream)
    if args.workload == "batch64":
        import synth as _s
        g0 = _s.powerlaw_10m(scale=args.scale)
        gg0 = tmg.Graph.from_synth(g0, device=dev, stream=stream)
        print(json.dumps({"workload": "batch64", "config": {"graph": g0.name, "delta_range_s": [60, 86400]},
                          "batched": batched_leg(gg0, dev, stream, dmax=86_400.0, autotune=False)}), flush=True)
        return
    g, queries = workload(args.scale, args.workload)
    count_only = args.workload == "hubskew_100m"
    m = g.n_edges
    with torch.cuda.stream(stream):
        gg = tmg.Graph.from_synth(g, device=dev, stream=stream)
        qs = [gg.compile(q) for q in queries]
        for q in qs:
            q.profile(True)
        # one 2^26-row buffer per query (the batched enumeration writes them all in one pass)
        outs = [torch.empty((1 if count_only else CAP, mo.k), dtype=torch.int32, device=f"cuda:{dev}")
                for mo in queries]
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")

        views = None if count_only else outs

        def step():
            # one search per query delivers both results: tm_enumerate_batch's count pass gives
            # each exact total (its per-chunk counts place the rows), its fill pass the rows
            if count_only:
                tot, kms = [], []
                for q in qs:
                    tot.append(q.count(stream=stream))
                    kms.append(q.last_ms()[0])
                return tot, kms, [0.0]
            _, tot, _, (cms, fms) = gg.enumerate_batch(qs, views, stream=stream, timed=True)
            return tot, [cms], [fms]

        for _ in range(args.warmup):
            step()
        totals = step()[0]
        # algorithm-independent work per query (untimed)
        works = [q.work(stream=stream) for q in qs]
        stream.synchronize()
        clocks = Clocks(dev)
        clocks.start()
        clocks.wait_samples(1)
        barrier(ws)
        torch.cuda.synchronize()
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        launches0 = tmg.kernel_launches()
        search_ms = []
        for s in range(args.steps):
            flush.zero_()                       # L2 flush between steps (outside the events)
            e0[s].record(stream)
            _, kms, fms = step()
            e1[s].record(stream)
            search_ms.append((kms, fms))
        torch.cuda.synchronize()
        launches = tmg.kernel_launches() - launches0 - 0
        barrier(ws)
        step_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
        clk = clocks.stop()
    ms = allmax(float(np.mean(step_ms)), ws)
    total_roots = len(queries) * m * ws
    value = total_roots / (ms / 1000.0)
    matches = sum(totals)
    # roofline of the dominant kernel: the count-mode search launch
    pk = peaks()
    count_ms = np.mean([sum(k) for k, _ in search_ms])      # count launches (tm_enumerate's count pass)
    fill_ms = np.mean([sum(f) for _, f in search_ms])
    lab = g.elabel is not None
    b_full = sum(alg_bytes(w, q.k, 0, lab)[0] for w, q in zip(works, queries))
    b_low = sum(alg_bytes(w, q.k, 0, lab)[1] for w, q in zip(works, queries))
    # achieved counts the bytes of the search itself (root columns, one sector per located
    # window, the window entries); the notional binary-search sectors of the full per-unit formula
    # are reported separately: with the successor index most windows need no search at all
    achieved = b_low / (count_ms / 1000.0) / 1e9
    launches_per_step = launches / args.steps
    line = {
        "metric": "root-edges/s", "value": value, "unit": "root-edges/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": step_config(g, queries, count_only, ws),
        "matches_per_s": matches * ws / (ms / 1000.0),
        "step_calls": "count only: tm_count per query" if count_only else
                      "one tm_enumerate_batch over the 4 queries: the exact totals from its count pass "
                      "(one persistent launch per occupancy group), the rows (capped at 2^26 per query) "
                      "from its fill pass",
        "totals": totals,
        "count_kernel_ms": ([round(float(np.mean([k[i] for k, _ in search_ms])), 4) for i in range(len(queries))]
                            if count_only else None),
        "count_pass_ms_per_step": round(float(count_ms), 4),
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"],
                     # DRAM bytes of one step's count pass, beside alg_bytes_per_step
                     "traffic": measured_traffic(args.workload) if args.scale == 1.0 else None,
                     # per query counted: the count pass runs one persistent launch per occupancy
                     # group, so achieved = the step's algorithmic bytes / the step's count time;
                     # traffic is the capture's DRAM bytes of one single-query count launch
                     "alg_bytes_per_query_count": int(b_low / len(queries)),
                     "kernel": "search_kernel<count>", "peak_source": pk["source"],
                     "with_notional_binary_search_GBps": b_full / (count_ms / 1000.0) / 1e9,
                     "alg_bytes_per_step": int(b_low),
                     "kernel_ms_per_step": {"count": count_ms, "fill": fill_ms}},
    }
    extras = rank == 0 and ws == 1 and not args.no_extras
    if extras:
        line["ablation"] = ablation_leg(queries, qs, stream)
    if extras and not count_only:
        line["e2e"] = e2e_leg(args, g, queries, dev)
        line["batched"] = batched_leg(gg, dev, stream)
        line["served"] = served_leg(gg, dev)
        line["cpu_baseline"] = cpu_leg(g, queries, args.cpu_seconds, count_only)
        for q in qs:
            q.free()
        gg.free()
        line["hubskew_100m"] = hubskew_leg(args, dev, stream, pk)
    elif extras:
        line["cpu_baseline"] = cpu_leg(g, queries, args.cpu_seconds, count_only)
    if rank == 0:
        print(json.dumps(line), flush=True)


def hubskew_leg(args, dev, stream, pk, reps=3):
    """The hub-skewed graph (100M edges, 10M nodes, Zipf 1.8 with 0.01% of nodes owning 20%
    of the endpoints, 16 edge labels, 30 days): counts of the labelled 5-edge path with gaps
    <= 600 s and of the chorded 4-cycle (delta 7200 s), each count launch timed with CUDA
    events, and the roofline of the pair (algorithmic bytes from the work counters)."""
    import torch
    import synth
    import paper_2310_02800_gb300 as tmg
    g = synth.hub_skewed_100m(scale=args.scale)
    queries = synth.hub_skewed_queries()
    with torch.cuda.stream(stream):
        gg = tmg.Graph.from_synth(g, device=dev, stream=stream)
        m = gg.n_edges
        rows, b_low, ms_sum = [], 0, 0.0
        for mo in queries:
            q = gg.compile(mo)
            q.profile(True)
            c = q.count(stream=stream)
            ms = []
            for _ in range(reps):
                assert q.count(stream=stream) == c
                ms.append(q.last_ms()[0])
            w = q.work(stream=stream)
            b = alg_bytes(w, mo.k, 0, True)[1]
            med = float(np.median(ms))
            b_low += b
            ms_sum += med
            rows.append({"query": mo.name, "matches": c, "count_ms": round(med, 3),
                         "alg_bytes": int(b), "root_edges_per_s": m / (med / 1000.0)})
            q.free()
        gg.free()
    achieved = b_low / (ms_sum / 1000.0) / 1e9
    return {"workload": g.name, "n_edges": m, "delta_s": queries[0].delta, "queries": rows,
            "root_edges_per_s": len(rows) * m / (ms_sum / 1000.0),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"], "kernel": "search_kernel<count>"}}


def sweeps(args, dev, stream, reps=3):
    """Constraint sweep (the paper's Table 4 shape: a temporal 4-cycle with no constraints, node
    labels, fine-grained gaps, an anti-edge) and the ablation against the paper's
    thread-per-tree baseline over delta (the shape of its Fig. 9), on the 10M-edge graph
    with two node labels."""
    import torch
    import synth
    import paper_2310_02800_gb300 as tmg
    g = synth.powerlaw_10m(scale=args.scale)
    g.nlabel = synth.node_labels(g.n_nodes, 2, synth.SEED_BASE + 6)
    out = {"workload": "sweeps", "config": {"graph": g.name, "node_labels": 2}}
    with torch.cuda.stream(stream):
        gg = tmg.Graph.from_synth(g, device=dev, stream=stream)
        rows = []
        for mo in synth.constraint_sweep_queries():
            q = gg.compile(mo)
            q.profile(True)
            c = q.count(stream=stream)
            ms = []
            for _ in range(reps):
                assert q.count(stream=stream) == c
                ms.append(q.last_ms()[0])
            rows.append({"query": mo.name, "matches": c, "count_ms": round(float(np.median(ms)), 4)})
        out["constraints"] = rows
        sweep = []
        for delta in (900, 1800, 3600, 7200):
            queries = synth.powerlaw_queries(delta)
            qs = [gg.compile(q) for q in queries]
            for q in qs:
                q.profile(True)
            for mo, r in ablation_leg(queries, qs, stream).items():
                sweep.append(dict(delta_s=delta, query=mo, **r))
        out["delta_sweep"] = sweep
    print(json.dumps(out), flush=True)


def ablation_leg(queries, qs, stream):
    """Same counts with the paper's thread-per-tree baseline design (Section 3.2) on this GPU."""
    out = {}
    for mo, q in zip(queries, qs):
        c0 = q.count(stream=stream)
        ms_ours = q.last_ms()[0]
        c1, ms_base = q.count_baseline(stream=stream)
        out[mo.name] = {"search_kernel_ms": round(ms_ours, 4), "baseline_kernel_ms": round(ms_base, 4),
                        "speedup": round(ms_base / max(ms_ours, 1e-9), 2), "counts_equal": c1 == c0}
    return out


def e2e_leg(args, g, queries, dev):
    """Public API with host buffers: graph upload + build, count + enumerate, match rows to host."""
    import torch
    import paper_2310_02800_gb300 as tmg
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    src, dst, t = pin(g.src), pin(g.dst), pin(g.t)
    host_rows = torch.empty((CAP, 4), dtype=torch.int32).pin_memory()
    # caller-owned row buffers, allocated once (as a user reuses them)
    outs = [torch.empty((CAP, mo.k), dtype=torch.int32, device=f"cuda:{dev}") for mo in queries]
    times, h2d, d2h = [], 0, 0
    phases = {"load": [], "enumerate_batch": [], "rows_to_host": [], "free": []}
    # host-timed: the median of 5 steps after 2 untimed ones, so one stall of the host does not
    # stand for the step
    for rep in range(2 + 5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gg = tmg.Graph.load(g.n_nodes, src, dst, t, device=dev)
        t1 = time.perf_counter()
        qs = [gg.compile(mo) for mo in queries]
        nws, tots, _ = gg.enumerate_batch(qs, outs)
        t2 = time.perf_counter()
        dbytes = 0
        for nw, out, mo in zip(nws, outs, queries):
            host_rows.view(-1)[: nw * mo.k].copy_(out[:nw].reshape(-1))
            dbytes += nw * mo.k * 4 + 8
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        for q in qs:
            q.free()
        gg.free()
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        dt = t4 - t0
        if rep >= 2:
            times.append(dt)
            for key, a, b in (("load", t0, t1), ("enumerate_batch", t1, t2), ("rows_to_host", t2, t3),
                              ("free", t3, t4)):
                phases[key].append(1000 * (b - a))
        d2h = dbytes
    h2d = g.n_edges * (4 + 4 + 8)
    sec = float(np.median(times))
    return {"value": len(queries) * g.n_edges / sec, "unit": "root-edges/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * sec,
            "phases_ms": {k: round(float(np.median(v)), 3) for k, v in phases.items()},
            "includes": "host->device upload and GPU build of the graph, one tm_enumerate_batch over the 4 "
                        "queries (exact counts + rows), rows to host"}


def mix_cost_sample(gg, mix, limit_s=1.0, max_frac=0.02, seed_stream=811, first_span=256):
    """Device seconds one full count of each query would take, extrapolated from root ranges
    at seeded positions (count only; each range's kernel time from CUDA events).  Ranges grow
    from first_span roots by doubling until 2% of the roots are covered or the query has used
    limit_s of wall time, so the cost of a query that would run for hours is found in about
    a second."""
    import synth
    m = gg.n_edges
    starts = [int(x) for x in synth.draws(synth.SEED_BASE + 4, seed_stream, 48)]
    rows = []
    for mo in mix:
        q = gg.compile(mo)
        q.profile(True)
        span, done, dev_ms, i = first_span, 0, 0.0, 0
        t0 = time.perf_counter()
        while done < max_frac * m and i < len(starts):
            span = min(span, m)
            a = starts[i] % max(1, m - span + 1)
            q.count_roots(a, a + span)
            dev_ms += q.last_ms()[0]
            done += span
            i += 1
            if time.perf_counter() - t0 > limit_s:
                break
            span *= 2
        rows.append({"query": mo.name, "est_s": dev_ms / 1000.0 * m / done, "sampled_roots": done})
        q.free()
    return rows


def batched_leg(gg, dev, stream, dmax=86_400.0, limit_s=2.0, reps=2, autotune=True):
    """Config of the batched workload: the seeded 64-query mix (k in 2..6, delta log-uniform in
    [60, dmax] s) counted in one CUDA-graph launch (one persistent launch per occupancy
    group) vs one query at a time.  Every query is first costed from a root sample; a query
    whose full count would take more than limit_s of device time is left out of both arms
    and reported with its estimate (the day-long 5- and 6-edge out-stars on this graph's hubs
    enumerate 1e11-1e13 matches).  Then, after per-shape autotuning of the cheap queries, both
    arms again."""
    import torch
    import synth
    mix = synth.query_mix(64, dmax=dmax)
    cost = mix_cost_sample(gg, mix)
    keep = [i for i, r in enumerate(cost) if r["est_s"] <= limit_s]
    left_out = [cost[i] for i in range(len(mix)) if i not in keep]
    qs = [gg.compile(mix[i]) for i in keep]
    m = gg.n_edges

    def timed(fn):
        t0 = time.perf_counter()
        for _ in range(reps):
            r = fn()
        return r, (time.perf_counter() - t0) / reps

    with torch.cuda.stream(stream):
        want = gg.count_batch(qs, stream=stream)
        got, tb = timed(lambda: gg.count_batch(qs, stream=stream))
        single, ts = timed(lambda: [q.count(stream=stream) for q in qs])
    n = len(qs)
    out = {"queries": len(mix), "timed_queries": n, "delta_range_s": [60, dmax],
           "left_out": left_out, "est_device_s_of_timed": sum(cost[i]["est_s"] for i in keep),
           "batched_ms": 1000 * tb, "sequential_ms": 1000 * ts,
           "batched_root_edges_per_s": n * m / tb, "sequential_root_edges_per_s": n * m / ts,
           "speedup": ts / tb, "totals_equal": got == want and single == want, "matches": int(sum(want))}
    if autotune:
        # per-shape tuning (warps per block, chunk size, split depth, split threshold) of the
        # queries that count in under 50 ms, untimed; the graph caches it by motif shape and
        # delta bucket, and both arms use it
        t0 = time.perf_counter()
        tuned = 0
        with torch.cuda.stream(stream):
            for q, i in zip(qs, keep):
                if cost[i]["est_s"] < 0.05:
                    q.autotune(stream=stream)
                    tuned += 1
            tune_s = time.perf_counter() - t0
            got2, tb2 = timed(lambda: gg.count_batch(qs, stream=stream))
            single2, ts2 = timed(lambda: [q.count(stream=stream) for q in qs])
        out["autotuned"] = {"tuned_queries": tuned, "batched_ms": 1000 * tb2, "sequential_ms": 1000 * ts2,
                            "speedup": ts2 / tb2, "vs_untuned_sequential": ts / tb2,
                            "vs_untuned_batched": tb / tb2, "tune_s": tune_s,
                            "totals_equal": got2 == want and single2 == want}
    return out


SERVE_RATES = ((50, 4000), (200, 4000), (1000, 4000), (2000, 4000), (5000, 4000))


def serve_trace(qs, kinds, rate, n, seed_stream):
    """(arrival s, query index, enumerate?) of n Poisson arrivals at `rate` q/s; 30% enumerate."""
    import synth
    arr = synth.arrival_trace(rate, n, synth.SEED_BASE + 5, stream=seed_stream)
    return [(float(arr[i]), i % len(qs), int(kinds[i % len(kinds)] % 10) < 3) for i in range(n)]


def run_served(gg, qs, reqs, cap, **shape):
    """Submit each request at its arrival time from one thread while a second thread
    collects results in submission order and releases them (a client that keeps results
    only as long as it needs them); latency = completion - scheduled arrival."""
    import queue
    srv = gg.serve(mem_budget_bytes=8 << 30, **shape)
    pending = queue.Queue()
    lat, totals = [], []

    def harvest():
        while True:
            item = pending.get()
            if item is None:
                return
            tk, lg = item
            r = srv.wait(tk)
            lat.append(1000.0 * lg + r.latency_ms)
            totals.append(r.total)
            srv.release(tk)

    th = threading.Thread(target=harvest)
    th.start()
    t0 = time.perf_counter()
    for at, qi, en in reqs:
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        lag = max(0.0, time.perf_counter() - t0 - at)
        pending.put((srv.submit(qs[qi], enumerate=en, cap=cap if en else 0), lag))
    pending.put(None)
    th.join()
    wall = time.perf_counter() - t0
    srv.stop()
    return lat, totals, wall


def run_serial(gg, qs, reqs, cap, dev):
    """One request at a time through tm_count / tm_enumerate, in arrival order (FIFO)."""
    import torch
    outbuf = torch.empty((cap, 6), dtype=torch.int32, device=f"cuda:{dev}")
    lat, totals = [], []
    t0 = time.perf_counter()
    for at, qi, en in reqs:
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        q = qs[qi]
        if en:
            _, tot, _ = q.enumerate(outbuf.view(-1)[: cap * q.k].view(cap, q.k))
        else:
            tot = q.count()
        totals.append(tot)
        lat.append(1000.0 * (time.perf_counter() - t0 - at))
    return lat, totals, time.perf_counter() - t0


def served_leg(gg, dev, dmax=3600.0, kmax=6, rates=SERVE_RATES, shape=None, cap=1_000_000, n_mix=256,
               progress=None):
    """Poisson arrivals of a 70% count / 30% enumerate mix (cap 1e6), k in 2..kmax, delta
    log-uniform in [60, dmax] s: served (continuous batching, the library's default shape
    unless `shape` is given) vs serial single-query execution of the same trace.  Latency runs
    from each request's scheduled arrival to its completion, in both arms; throughput =
    requests / wall time from the first arrival to the last completion."""
    import synth
    shape = shape or {}
    mix = synth.query_mix(n_mix, seed=synth.SEED_BASE + 5, dmax=dmax, kmax=kmax)
    kinds = synth.draws(synth.SEED_BASE + 5, 601, n_mix)
    qs = [gg.compile(q) for q in mix]
    out = {"delta_range_s": [60, dmax], "k_range": [2, kmax], "mix": "70% count / 30% enumerate (cap 1e6)",
           "shape": shape or "library default (2 streams, batches by expected cost)"}
    # one untimed pass over the mix: compiled queries warm, and the graph's per-shape cost
    # estimates (kept by the library for every server of this graph) learnt
    warm = serve_trace(qs, kinds, 1e9, len(qs), 699)
    run_served(gg, qs, warm, cap, **shape)
    for rate, n in rates:
        # one draw stream per rate (rates below 1 q/s get their own range)
        reqs = serve_trace(qs, kinds, rate, n, 700 + int(rate) if rate >= 1 else 690 + int(rate * 20))
        lat, tot_a, wall = run_served(gg, qs, reqs, cap, **shape)
        slat, tot_b, swall = run_serial(gg, qs, reqs, cap, dev)
        out[str(rate)] = {"requests": n, "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99)), "throughput_qps": n / wall,
                          "serial_p50_ms": float(np.percentile(slat, 50)),
                          "serial_p99_ms": float(np.percentile(slat, 99)), "serial_throughput_qps": n / swall,
                          "root_edges_per_s": gg.n_edges * n / wall, "results_equal": tot_a == tot_b}
        if progress:
            progress(phase="served", rate=rate, **out[str(rate)])
    return out


def powerlaw_1b_graph(scale):
    """The 1B-edge, 100M-node graph (Zipf 2.1 popularity on both endpoints)."""
    import synth
    return synth.powerlaw_1b(scale=scale)


def count_1b(args, dev, stream, delta=600):
    """GPU ingest of the 1B-edge graph from host arrays, then counts of the four power-law
    queries (delta 600 s: longer windows on this graph's hubs make single counts run for
    minutes)."""
    import torch
    import synth
    import paper_2310_02800_gb300 as tmg
    t0 = time.perf_counter()
    g = powerlaw_1b_graph(args.scale)
    gen_s = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        gg = tmg.Graph.from_synth(g, device=dev, stream=stream)
        torch.cuda.synchronize()
        load_s = time.perf_counter() - t0
        m = gg.n_edges
        del g
        queries = synth.powerlaw_queries(delta)
        qs = [gg.compile(q) for q in queries]
        rows = []
        for mo, q in zip(queries, qs):
            q.profile(True)
            c = q.count(stream=stream)
            ms = []
            for _ in range(max(1, args.steps)):
                assert q.count(stream=stream) == c
                ms.append(q.last_ms()[0])
            rows.append({"query": mo.name, "matches": c, "count_ms": round(float(np.median(ms)), 2),
                         "root_edges_per_s": m / (float(np.median(ms)) / 1000.0)})
    total_ms = sum(r["count_ms"] for r in rows)
    print(json.dumps({"metric": "root-edges/s", "value": len(rows) * m / (total_ms / 1000.0), "unit": "root-edges/s",
                      "workload": "count_1b",
                      "config": {"graph": f"powerlaw_1b x{args.scale}", "n_edges": m, "n_nodes": gg.n_nodes,
                                 "delta_s": delta, "device_bytes": gg.device_bytes, "generate_s": gen_s,
                                 "upload_and_build_s": load_s},
                      "queries": rows}), flush=True)


def serve_1b(args, dev):
    """The serving workload on the resident 1B-edge graph: the part of the stated mix a
    latency trace can absorb (k 2..4, delta <= 600 s; the day-window stars of the stated mix
    enumerate over 1e13 matches per request on the 10M-edge graph already, and a single hub
    root of them on this graph over 1e15) is first timed request by request, then served at
    Poisson rates around its capacity against serial execution of the same trace.  Each
    phase reports on stderr as it ends."""
    import synth
    import paper_2310_02800_gb300 as tmg

    def note(**kw):
        print(json.dumps(kw), file=sys.stderr, flush=True)

    t0 = time.perf_counter()
    g = powerlaw_1b_graph(args.scale)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    gg = tmg.Graph.from_synth(g, device=dev)
    load_s = time.perf_counter() - t0
    del g
    note(phase="loaded", generate_s=gen_s, load_s=load_s, device_bytes=gg.device_bytes)
    mix = synth.query_mix(16, seed=synth.SEED_BASE + 5, dmax=600.0, kmax=4)
    cost = []
    for mo in mix:
        q = gg.compile(mo)
        q.profile(True)
        c = q.count()
        cost.append({"query": mo.name, "count_ms": q.last_ms()[0], "matches": c})
        q.free()
    note(phase="costed", rows=cost)
    res = served_leg(gg, dev, dmax=600.0, kmax=4, rates=((0.25, 16), (1.0, 32)), n_mix=16, progress=note)
    line = {"metric": "p50/p99 latency and throughput, served vs serial", "workload": "serve_1b",
            "config": {"workload": f"powerlaw_1b x{args.scale}", "n_edges": gg.n_edges, "n_nodes": gg.n_nodes,
                       "device_bytes": gg.device_bytes, "generate_s": gen_s, "load_s": load_s},
            "mix_count_ms": cost, "served": res}
    print(json.dumps(line), flush=True)


def cpu_leg(g, queries, seconds, count_only=False):
    """The oracle timed on the host's cores: root-range parallel over all of them (the
    baseline), and on one core beside it."""
    import oracle
    og = oracle.Graph.from_synth(g)
    cores = host_cores()
    rate, spent, roots = oracle_rate(g, queries, seconds, cores, count_only, og)
    rate1, spent1, roots1 = oracle_rate(g, queries, seconds / 3, 1, count_only, og)
    what = "counted" if count_only else "counted and enumerated"
    return {"value": rate, "unit": "root-edges/s", "cores": cores, "kind": "oracle",
            "sample": f"{roots} root edges in contiguous ranges of the {len(queries)} queries, {what}, "
                      f"split into {cores} root ranges on {cores} threads ({spent:.1f} s)",
            "nproc": os.cpu_count(),
            "single_core": {"value": rate1, "unit": "root-edges/s", "cores": 1,
                            "sample": f"{roots1} root edges, {what} ({spent1:.1f} s)"}}


if __name__ == "__main__":
    main()
