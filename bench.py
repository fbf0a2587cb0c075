"""Benchmark: temporal motif mining on one GB300 (or N replicas under torchrun).

Default workload (one "step"): the 10M-edge power-law temporal graph (1M
nodes, Zipf 2.1, bursty 3-year timestamps, 10% reciprocated edges), resident in
HBM; each of its four queries (3-cycle, 4-cycle, 3-edge out-star, 4-edge
ping-pong; delta = 3600 s) is counted (tm_count) and enumerated into a
2^26-row buffer (tm_enumerate).  value = root-edges/s = 4 queries x m roots /
step time.  Extra objects on the same line: matches/s, the batched form
(64-query mix in one CUDA-graph launch vs 64 single launches), the served form
(Poisson arrivals, p50/p99 vs serial single-query execution), the roofline of
the dominant kernel and the CPU oracle baseline.

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

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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

def oracle_rate(g, queries, seconds, og=None):
    """Oracle count over contiguous root ranges of every query, grown until ~seconds of CPU work."""
    import oracle
    og = og or oracle.Graph.from_synth(g)
    m = g.n_edges
    roots = 2048
    spent = 0.0
    done_roots = 0
    while True:
        t0 = time.perf_counter()
        for qi, q in enumerate(queries):
            a = (m // (len(queries) + 1)) * (qi + 1)
            og.count(q, a, min(m, a + roots))
        dt = time.perf_counter() - t0
        spent += dt
        done_roots += roots * len(queries)
        if spent >= seconds or roots >= m:
            break
        roots = min(m, int(roots * max(2.0, min(8.0, seconds / max(dt, 1e-3)))))
        if spent + dt * 8 > seconds * 1.5:
            roots = min(roots, int(roots / 4) + 1)
    return done_roots / spent, spent, done_roots


def run_reference(args, rank, ws):
    if rank != 0:
        return
    g, queries = workload(args.scale, args.workload)
    import oracle
    t0 = time.perf_counter()
    og = oracle.Graph.from_synth(g)
    build_s = time.perf_counter() - t0
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    times, roots_total = [], 0
    for s in range(args.warmup + args.steps):
        rate, spent, roots = oracle_rate(g, queries, per_step, og)
        if s >= args.warmup:
            times.append(spent)
            roots_total += roots
    value = roots_total / sum(times)
    line = {"impl": "reference", "metric": "root-edges/s", "value": value, "unit": "root-edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": g.name, "queries": [q.name for q in queries], "delta_s": 3600},
            "cpu_baseline": {"value": value, "unit": "root-edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"contiguous root ranges of each query, ~{per_step:.0f} s of CPU per step; "
                                       f"oracle graph build {build_s:.1f} s not timed"},
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
    """DRAM bytes per count launch from the committed ncu capture of this kernel on this
    workload; None when the kernel sources changed since it was taken."""
    if workload != "powerlaw_10m" or not os.path.exists(TRAFFIC_FILE):
        return None
    d = json.load(open(TRAFFIC_FILE))
    if d.get("kernel_source_sha256") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_count_launch"])


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
        out = torch.empty((1 if count_only else CAP, max(q.k for q in queries)), dtype=torch.int32,
                          device=f"cuda:{dev}")
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")

        def step():
            tot, kms, fms = [], [], []
            for mo, q in zip(queries, qs):
                c = q.count(stream=stream)
                kms.append(q.last_ms()[0])
                if not count_only:
                    view = out.view(-1)[: CAP * mo.k].view(CAP, mo.k)
                    nw, t2, _ = q.enumerate(view, stream=stream)
                    a, b = q.last_ms()
                    kms.append(a); fms.append(b)
                    assert t2 == c
                else:
                    kms.append(0.0); fms.append(0.0)
                tot.append(c)
            return tot, kms, fms

        for _ in range(args.warmup):
            step()
        totals = step()[0]
        # algorithm-independent work per query (untimed)
        works = [q.work(stream=stream) for q in qs]
        stream.synchronize()
        clocks = Clocks(dev)
        clocks.start()
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
    count_ms = np.mean([sum(k[0::2]) for k, _ in search_ms])     # count pass of tm_count per query
    fill_ms = np.mean([sum(f) for _, f in search_ms])
    enum_count_ms = np.mean([sum(k[1::2]) for k, _ in search_ms])
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
        "config": {"workload": g.name, "n_nodes": g.n_nodes, "n_edges": m,
                   "queries": [q.name for q in queries], "delta_s": queries[0].delta,
                   "enumerate_cap": None if count_only else CAP,
                   "step": "count of each query" if count_only else "count + capped enumerate of each query",
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}"},
        "matches_per_s": matches * ws / (ms / 1000.0),
        "totals": totals,
        "count_kernel_ms": [round(float(np.mean([k[2 * i] for k, _ in search_ms])), 4) for i in range(len(queries))],
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"],
                     "traffic": measured_traffic(args.workload) if args.scale == 1.0 else None,
                     "alg_bytes_per_launch": int(b_low / len(queries)),
                     "kernel": "search_kernel<count>", "peak_source": pk["source"],
                     "with_notional_binary_search_GBps": b_full / (count_ms / 1000.0) / 1e9,
                     "alg_bytes_per_step": int(b_low),
                     "kernel_ms_per_step": {"count": count_ms, "enum_count_pass": enum_count_ms, "fill": fill_ms}},
    }
    if rank == 0 and not args.no_extras:
        line["ablation"] = ablation_leg(queries, qs, stream)
    if rank == 0 and not args.no_extras and not count_only:
        line["e2e"] = e2e_leg(args, g, queries, dev)
        line["batched"] = batched_leg(gg, dev, stream)
        line["served"] = served_leg(gg, dev)
        line["cpu_baseline"] = cpu_leg(g, queries, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)


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
    times, h2d, d2h = [], 0, 0
    for rep in range(2 + max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gg = tmg.Graph.load(g.n_nodes, src, dst, t, device=dev)
        dbytes = 0
        for mo in queries:
            q = gg.compile(mo)
            q.count()
            out = torch.empty((CAP, mo.k), dtype=torch.int32, device=f"cuda:{dev}")
            nw, tot, _ = q.enumerate(out)
            host_rows.view(-1)[: nw * mo.k].copy_(out[:nw].reshape(-1))
            dbytes += nw * mo.k * 4 + 8
            q.free()
        gg.free()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if rep >= 2:
            times.append(dt)
        d2h = dbytes
    h2d = g.n_edges * (4 + 4 + 8)
    sec = float(np.mean(times))
    return {"value": len(queries) * g.n_edges / sec, "unit": "root-edges/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * sec,
            "includes": "host->device upload and GPU build of the graph, 4x(count + enumerate), rows to host"}


def batched_leg(gg, dev, stream, dmax=3600.0, autotune=True):
    """64-query mix (k in 2..6, delta log-uniform in [60, dmax]): one persistent CUDA-graph
    launch vs 64 single-query launches.  The default dmax keeps the leg to seconds; the full
    [60, 86400] range is --workload batch64."""
    import torch
    import synth
    mix = synth.query_mix(64, dmax=dmax)
    qs = [gg.compile(q) for q in mix]
    with torch.cuda.stream(stream):
        want = gg.count_batch(qs, stream=stream)
        for _ in range(2):
            gg.count_batch(qs, stream=stream)
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            got = gg.count_batch(qs, stream=stream)
        tb = (time.perf_counter() - t0) / reps
        assert got == want
        single = [q.count(stream=stream) for q in qs]
        t0 = time.perf_counter()
        for _ in range(reps):
            single = [q.count(stream=stream) for q in qs]
        ts = (time.perf_counter() - t0) / reps
    ok = single == want
    m = gg.n_edges
    out = {"queries": 64, "delta_range_s": [60, dmax], "batched_ms": 1000 * tb, "sequential_ms": 1000 * ts,
           "batched_root_edges_per_s": 64 * m / tb, "sequential_root_edges_per_s": 64 * m / ts,
           "speedup": ts / tb, "totals_equal": ok, "matches": int(sum(want))}
    if autotune:
        # per-shape tuning (warps per block, chunk size, split depth, split threshold), untimed;
        # the graph caches it by motif shape and delta bucket for later compiles
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for q in qs:
                q.autotune(stream=stream)
            tune_s = time.perf_counter() - t0
            gg.count_batch(qs, stream=stream)
            t0 = time.perf_counter()
            for _ in range(reps):
                got = gg.count_batch(qs, stream=stream)
            tb2 = (time.perf_counter() - t0) / reps
            t0 = time.perf_counter()
            for _ in range(reps):
                single = [q.count(stream=stream) for q in qs]
            ts2 = (time.perf_counter() - t0) / reps
        out["autotuned"] = {"batched_ms": 1000 * tb2, "sequential_ms": 1000 * ts2, "speedup": ts2 / tb2,
                            "vs_untuned_sequential": ts / tb2, "tune_s": tune_s,
                            "totals_equal": got == want and single == want}
    return out


def served_leg(gg, dev, duration_s=2.0, dmax=3600.0, max_requests=400, kmax=6,
               shapes=((2, 16), (1, 16), (2, 4), (2, 1), (4, 4), (4, 1))):
    """Poisson arrivals (50 / 200 / 1000 q/s) of a 70% count / 30% enumerate mix (cap 1e6),
    k in 2..6, delta log-uniform in [60, dmax]: served (continuous batching) vs serial
    single-query execution of the same trace."""
    import torch
    import synth
    out = {"delta_range_s": [60, dmax], "k_range": [2, kmax]}
    mix = synth.query_mix(256, seed=synth.SEED_BASE + 5, dmax=dmax, kmax=kmax)
    kinds = synth.draws(synth.SEED_BASE + 5, 601, 256)
    qs = [gg.compile(q) for q in mix]
    for rate in (50, 200, 1000):
        n = min(max_requests, max(8, int(rate * duration_s)))
        arr = synth.arrival_trace(rate, n, synth.SEED_BASE + 5, stream=700 + rate)
        reqs = [(float(arr[i]), i % len(qs), int(kinds[i % len(kinds)] % 10) < 3) for i in range(n)]
        configs = {}
        for streams, max_batch in shapes:
            srv = gg.serve(mem_budget_bytes=8 << 30, streams=streams, max_batch=max_batch)
            lat, tickets = [], []
            t0 = time.perf_counter()
            for at, qi, en in reqs:
                now = time.perf_counter() - t0
                if at > now:
                    time.sleep(at - now)
                tickets.append(srv.submit(qs[qi], enumerate=en, cap=1_000_000 if en else 0))
            for tk in tickets:
                r = srv.wait(tk)
                lat.append(r.latency_ms)
                srv.release(tk)
            wall = time.perf_counter() - t0
            srv.stop()
            configs[f"streams{streams}_batch{max_batch}"] = {
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "throughput_qps": n / wall}
        # serial single-query execution of the same trace (FIFO, one at a time)
        slat = []
        outbuf = torch.empty((1_000_000, 6), dtype=torch.int32, device=f"cuda:{dev}")
        t0 = time.perf_counter()
        busy_until = 0.0
        for at, qi, en in reqs:
            now = time.perf_counter() - t0
            if at > now and at > busy_until:
                time.sleep(at - now)
            s0 = time.perf_counter() - t0
            q = qs[qi]
            if en:
                q.enumerate(outbuf.view(-1)[: 1_000_000 * q.k].view(1_000_000, q.k))
            else:
                q.count()
            done = time.perf_counter() - t0
            busy_until = done
            slat.append(1000 * (done - at))
        swall = time.perf_counter() - t0
        m = gg.n_edges
        # headline: the library's default shape (2 streams, batches of up to 16), chosen before
        # the run; the lowest p99 over all shapes tried is reported beside it
        main = f"streams{shapes[0][0]}_batch{shapes[0][1]}"
        best = min(configs, key=lambda c: (configs[c]["p99_ms"], -configs[c]["throughput_qps"]))
        out[str(rate)] = {"requests": n, "shape": main, **configs[main], "best_shape": best,
                          "best_shape_p99_ms": configs[best]["p99_ms"],
                          "root_edges_per_s": m * configs[main]["throughput_qps"],
                          "serial_p50_ms": float(np.percentile(slat, 50)), "serial_p99_ms": float(np.percentile(slat, 99)),
                          "serial_throughput_qps": n / swall, "configs": configs}
    return out


def powerlaw_1b_graph(scale):
    """The 1B-edge, 100M-node graph: Zipf 2.1 popularity on both endpoints (no copy model:
    at 1e9 edges preferential attachment puts ~15% of all edges on one node)."""
    import synth
    n = max(16, int(100_000_000 * scale)); m = max(16, int(1_000_000_000 * scale))
    return synth.powerlaw_graph(n, m, synth.SEED_BASE + 5, alpha=2.1, span=94_608_000.0, pa=False)


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
    """Served Poisson traces on the resident 1B-edge power-law graph."""
    import synth
    import paper_2310_02800_gb300 as tmg
    t0 = time.perf_counter()
    g = powerlaw_1b_graph(args.scale)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    gg = tmg.Graph.from_synth(g, device=dev)
    load_s = time.perf_counter() - t0
    del g
    # 2-4 edges, delta up to 10 minutes: longer windows on this graph's hubs make single
    # requests run for minutes, which a latency trace cannot absorb
    res = served_leg(gg, dev, duration_s=2.0, dmax=600.0, max_requests=40, kmax=4, shapes=((2, 16), (4, 4)))
    line = {"metric": "p50/p99 latency and throughput, served vs serial", "workload": gg.n_edges,
            "config": {"workload": f"powerlaw_1b x{args.scale}", "n_edges": gg.n_edges, "n_nodes": gg.n_nodes,
                       "device_bytes": gg.device_bytes, "generate_s": gen_s, "load_s": load_s},
            "served": res}
    print(json.dumps(line), flush=True)


def cpu_leg(g, queries, seconds):
    rate, spent, roots = oracle_rate(g, queries, seconds)
    return {"value": rate, "unit": "root-edges/s", "cores": 1, "kind": "oracle",
            "sample": f"{roots} root edges over contiguous ranges of the 4 queries ({spent:.1f} s single-threaded)"}


if __name__ == "__main__":
    main()
