#!/usr/bin/env python3
"""Benchmark of exact butterfly counting on one GB300 (or N replicas).

Step = one pass of the whole single-graph hot path over one synthetic graph:
prepare (degrees, priority ranks, projection + sorted lists, cut/work,
schedule) followed by the wedge count and its reduction, with the CSR already
resident in HBM.  Metric: processed wedges per second (W per step divided by
the device time of the step).  Also reported: the count kernel against the
HBM roofline, the CPU oracle timed on the host, and an end-to-end number
through the C ABI from host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload powerlaw_20m|shopping_300m|uniform_small]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "wedges/s & %HBM roofline (1 graph); graphs/s and p99 latency batched vs per-graph"
UNIT = "wedges/s"
L2_FLUSH_BYTES = 512 << 20
# the largest single-GPU workload, specified with per-vertex and per-edge counts
HEADLINE = "shopping_300m"
WORKLOADS = {
    "powerlaw_20m": "chunglu_u1m_l500k_m20m_g2.1 (|U|=1M, |L|=500k, 20M edges, exponent 2.1 both layers, seed 2001+rank)",
    "shopping_300m": "shopping_u10m_l100k_m300m (users exponent 2.5, items exponent 1.8, top item ~1M, seed 3001+rank)",
    "uniform_small": "uniform_u2k_l3k_m20k (seed 1001+rank)",
    "serve_poisson": "Poisson request stream: graphs drawn as the batched workload (pool of 256, seeds 5001+i) plus 2% large graphs (5M edges, exponent 2.0, |U|=1M, |L|=500k); 120 GB admission budget",
    "batch_4096": "4,096 Chung-Lu graphs, |U|,|L| log-uniform [100, 50k], m log-uniform [1k, 2M] clamped to 0.5|U||L|, exponents uniform [1.8, 2.6], seeds 4000+g (+rank*4096)",
}


def make_graph(name: str, rank: int, device):
    from bfc_inputs import generators as G
    if name == "powerlaw_20m":
        return G.powerlaw_20m(seed=2001 + rank, device=device)
    if name == "shopping_300m":
        return G.shopping_300m(seed=3001 + rank, device=device)
    if name == "uniform_small":
        return G.uniform_small(seed=1001 + rank, device=device)
    raise SystemExit(f"unknown workload {name}")


def run_batch(args, rank, world):
    """The batched workload: every graph of the batch counted per step, as
    one prepare over the disjoint union + one persistent count launch; the
    per-graph path (one prepare + one count per graph) timed beside it."""
    import numpy as np
    import torch

    from bfc_inputs import generators as G
    from paper_1812_00283_gb300 import bfc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, dev)
    num = args.batch_graphs
    t0 = time.perf_counter()
    graphs = [G.batch_graph(g, 4000 + rank * num, device=dev) for g in range(num)]
    b = G.union_batch(graphs)
    gen_s = time.perf_counter() - t0
    s = torch.cuda.current_stream()
    sp = s.cuda_stream
    off = torch.from_numpy(b.union.off_u).to(dev)
    adj = torch.from_numpy(b.union.adj_u).to(dev)
    us = torch.from_numpy(b.u_start).to(dev)
    ls = torch.from_numpy(b.l_start).to(dev)
    r, l, m = b.union.num_u, b.union.num_l, b.union.num_edges
    tots = torch.zeros(num, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # autotune the bin thresholds once on this batch (untimed)
    h = bfc.bfc_prepare_batch(r, l, m, off.data_ptr(), adj.data_ptr(), num, us.data_ptr(),
                              ls.data_ptr(), None, sp)
    chosen = bfc.bfc_autotune(h, sp, 2)
    opts = bfc.bfc_options_init(warp_max_work=chosen.warp_max_work, team_max_work=chosen.team_max_work,
                                hash_max_work=chosen.hash_max_work)
    bfc.bfc_count_batch(h, sp, tots.data_ptr(), None)
    wed = torch.zeros(num, dtype=torch.int64, device=dev)
    bfc.bfc_batch_wedges(h, sp, wed.data_ptr())
    torch.cuda.synchronize()
    expect = tots.clone()
    W = int(wed.sum().item())
    # count-only replay of a CUDA-graph capture of the batched count launch
    cg = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(s)
    with torch.cuda.graph(cg, stream=cap):
        bfc.bfc_count_batch(h, cap.cuda_stream, tots.data_ptr(), None)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cg.replay()
    e0.record(s)
    for _ in range(3):
        cg.replay()
    e1.record(s)
    torch.cuda.synchronize()
    graph_count_ms = e0.elapsed_time(e1) / 3
    if not torch.equal(tots, expect):
        raise SystemExit("graph replay changed the per-graph totals")
    bfc.bfc_release(h)

    def step(ev=None):
        if ev:
            ev[0].record(s)
        hh = bfc.bfc_prepare_batch(r, l, m, off.data_ptr(), adj.data_ptr(), num, us.data_ptr(),
                                   ls.data_ptr(), opts, sp)
        bfc.bfc_count_batch(hh, sp, tots.data_ptr(), None)
        bfc.bfc_release(hh)
        if ev:
            ev[1].record(s)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    props = torch.cuda.get_device_properties(dev)
    clk = ClockSampler(f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local))
    launches0 = bfc.bfc_kernel_launches()
    dist_barrier(world)
    torch.cuda.synchronize()
    clk.start()
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        step(evs[i])
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = bfc.bfc_kernel_launches() - launches0
    dist_barrier(world)
    if not torch.equal(tots, expect):
        raise SystemExit("per-graph totals changed between steps")
    step_ms = [e[0].elapsed_time(e[1]) for e in evs]
    t_total, graphs_all, (p50_all, p99_all) = reduce_over_ranks(
        world, dev, sum(step_ms), num * args.steps, (statistics.median(step_ms), max(step_ms)))
    _, W_all, _ = reduce_over_ranks(world, dev, 0.0, W * args.steps)
    value = graphs_all / (t_total / 1e3)

    # the whole step (a1-a7: checks, ranks, projection, cut/work, bins, the
    # persistent count, per-graph totals) recorded once as a CUDA graph on a
    # batch plan and replayed: no host synchronisation and no allocation per
    # step (tuned bounds as above)
    max_layer = max(max(g.num_u, g.num_l) for g in graphs)
    plan = bfc.bfc_batch_plan_create(r, l, m, num, max_layer, opts, sp)
    ptot = torch.zeros(num, dtype=torch.int64, device=dev)
    pst = torch.zeros(1, dtype=torch.int32, device=dev)
    bfc.bfc_batch_plan_run(plan, off.data_ptr(), adj.data_ptr(), us.data_ptr(), ls.data_ptr(), sp,
                           ptot.data_ptr(), pst.data_ptr())
    torch.cuda.synchronize()
    pg = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(s)
    with torch.cuda.graph(pg, stream=cap):
        bfc.bfc_batch_plan_run(plan, off.data_ptr(), adj.data_ptr(), us.data_ptr(), ls.data_ptr(),
                               cap.cuda_stream, ptot.data_ptr(), pst.data_ptr())
    for _ in range(args.warmup):
        flush.fill_(1)
        pg.replay()
    pevs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        pevs[i][0].record(s)
        pg.replay()
        pevs[i][1].record(s)
    torch.cuda.synchronize()
    if int(pst.item()) != 0 or not torch.equal(ptot, expect):
        raise SystemExit("the batch plan's replayed step disagrees with the batched path")
    plan_ms = [e[0].elapsed_time(e[1]) for e in pevs]
    bfc.bfc_batch_plan_destroy(plan)
    del pg

    # the per-graph path: one prepare + one count launch per graph, in turn
    lat = []
    done_at = []
    got = []
    dev_graphs = [(torch.from_numpy(g.off_u).to(dev), torch.from_numpy(g.adj_u).to(dev)) for g in graphs]
    one = torch.zeros(1, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    tp0 = time.perf_counter()
    for g, (o, a) in zip(graphs, dev_graphs):
        ta = time.perf_counter()
        hh = bfc.bfc_prepare(g.num_u, g.num_l, g.num_edges, o.data_ptr(), a.data_ptr(), opts, sp)
        bfc.bfc_count(hh, sp, one.data_ptr())
        bfc.bfc_release(hh)
        got.append(int(one.item()))
        tb = time.perf_counter()
        lat.append(tb - ta)
        done_at.append(tb - tp0)
    per_graph_s = time.perf_counter() - tp0
    if got != [int(x) for x in expect.cpu().numpy().view(np.uint64)]:
        raise SystemExit("per-graph path disagrees with the batched path")
    lat_ms = sorted(1e3 * x for x in lat)
    done_ms = sorted(1e3 * x for x in done_at)

    def pct(p, xs=None):
        xs = lat_ms if xs is None else xs
        return xs[min(len(xs) - 1, int(round(p / 100 * (len(xs) - 1))))]

    out = dict(
        metric=METRIC, value=value, unit="graphs/s", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=t_total / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="u64", data="synthetic",
        config=dict(workload=WORKLOADS["batch_4096"], num_graphs=num, union_edges=m,
                    wedges_per_step=W, step="prepare over the union (a1-a5) + one persistent count launch (a6-a7)",
                    l2="flushed between steps (512 MB write outside the timed events)",
                    autotuned=dict(warp_max_work=chosen.warp_max_work, team_max_work=chosen.team_max_work,
                                   hash_max_work=chosen.hash_max_work),
                    parallelism=f"replicas x{world} (each rank its own batch, no collective)",
                    generation_s=gen_s),
        plan_graph_replay=dict(graphs_per_s=num / (statistics.median(plan_ms) / 1e3),
                               ms_per_step_median=statistics.median(plan_ms), ms_per_step_max=max(plan_ms),
                               note="the whole step (checks, ranks, projection, cut/work, bins, count, "
                                    "per-graph totals) as one CUDA graph replay of a batch plan: no host "
                                    "synchronisation, no allocation; totals equal the batched path's"),
        batched=dict(graphs_per_s=value, wedges_per_s=W_all / (t_total / 1e3),
                     latency_ms_p50=p50_all, latency_ms_p99=p99_all,
                     request_completion_ms_p50=p50_all, request_completion_ms_p99=p99_all,
                     count_only_cuda_graph_ms=graph_count_ms,
                     note="every request of the batch completes when its step ends: a request's "
                          "latency from the batch's arrival is the step time"),
        per_graph=dict(graphs_per_s=num / per_graph_s, latency_ms_p50=pct(50), latency_ms_p99=pct(99),
                       request_completion_ms_p50=pct(50, done_ms), request_completion_ms_p99=pct(99, done_ms),
                       note="bfc_prepare + bfc_count + host read of the total, one graph at a time; "
                            "latency_ms = one graph alone, request_completion_ms = from the arrival of "
                            "the whole batch at once (like for like with the batched step)"),
        gpu_launches=launches, clocks=clocks)
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist_done(world)
    return 0


def run_serve(args, rank, world):
    """Serving: a Poisson stream of counting requests at swept arrival rates,
    through the continuous-batching server and through plain per-graph
    launches (a server with one worker and one graph per batch)."""
    import random

    import numpy as np
    import torch

    from bfc_inputs import generators as G
    from paper_1812_00283_gb300 import bfc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, dev)
    t0 = time.perf_counter()
    pool = [G.batch_graph(i, 5001 + rank * 1000, device=dev) for i in range(args.serve_pool)]
    large = [G.chung_lu_bipartite(1_000_000, 500_000, 5_000_000, 2.0, 2.0, 5900 + rank * 10 + i,
                                  device=dev) for i in range(max(1, args.serve_pool // 50))]
    gen_s = time.perf_counter() - t0
    arrays = [(np.ascontiguousarray(g.off_u), np.ascontiguousarray(g.adj_u)) for g in pool + large]
    rng = random.Random(5001 + rank)
    nreq = args.serve_requests
    # 2% of the requests are large graphs
    choice = [(len(pool) + rng.randrange(len(large))) if rng.random() < 0.02 else rng.randrange(len(pool))
              for _ in range(nreq)]
    gs = pool + large

    def serve(cfg, rate):
        """Submit the stream at `rate` requests/s (inf = all at once); returns
        (graphs/s over the makespan, latencies in ms, totals, stats)."""
        sv = bfc.bfc_server_create(cfg)
        ids = [0] * nreq
        arr = np.cumsum([rng2.expovariate(rate) for _ in range(nreq)]) if rate != float("inf") else np.zeros(nreq)
        try:
            tstart = time.perf_counter()

            def submit():
                for j, gi in enumerate(choice):
                    wait = tstart + arr[j] - time.perf_counter()
                    if wait > 0:
                        time.sleep(wait)
                    g = gs[gi]
                    off, adj = arrays[gi]
                    ids[j] = bfc.bfc_server_submit(sv, g.num_u, g.num_l, g.num_edges,
                                                   off.ctypes.data, adj.ctypes.data)
            th = threading.Thread(target=submit)
            th.start()
            th.join()
            res = [bfc.bfc_server_poll(sv, rid, True) for rid in ids]
            makespan = time.perf_counter() - tstart
            stats = bfc.bfc_server_get_stats(sv)
        finally:
            bfc.bfc_server_destroy(sv)
        if any(st != 0 for st, _, _ in res):
            raise SystemExit("a served request failed")
        lat = sorted(1e3 * x for _, _, x in res)
        return nreq / makespan, lat, [t for _, t, _ in res], stats

    def pct(lat, p):
        return lat[min(len(lat) - 1, int(round(p / 100 * (len(lat) - 1))))]

    rng2 = random.Random(17)
    batched_cfg = bfc.bfc_server_config_init(memory_budget_bytes=120 << 30, workers=2)
    plain_cfg = bfc.bfc_server_config_init(memory_budget_bytes=120 << 30, workers=1, max_batch_graphs=1)
    # warm-up: pool + kernels
    serve(batched_cfg, float("inf"))
    dist_barrier(world)
    sat_b, lat_b, tot_b, st_b = serve(batched_cfg, float("inf"))
    sat_p, lat_p, tot_p, st_p = serve(plain_cfg, float("inf"))
    dist_barrier(world)
    if tot_b != tot_p:
        raise SystemExit("served totals differ between batched and plain serving")
    rates = []
    # arrival rates as fractions of the batched server's saturation, plus
    # rates both servers sustain (fractions of the per-graph server's), where
    # the two p99 latencies compare like for like
    sweep = [(f * sat_b, f, "batched") for f in args.serve_rates] + \
            [(f * sat_p, f, "per_graph") for f in args.serve_rates_per_graph]
    for lam, frac, ref in sweep:
        gb, lb, tb, sb = serve(batched_cfg, lam)
        gp, lp, tp, sp_ = serve(plain_cfg, lam) if lam <= 1.5 * sat_p else (None, None, None, None)
        if tb != tot_b or (tp is not None and tp != tot_b):
            raise SystemExit("a served total changed with the arrival rate")
        row = dict(rate_per_s=lam, **{f"frac_of_{ref}_saturation": frac},
                   batched=dict(graphs_per_s=gb, p50_ms=pct(lb, 50), p99_ms=pct(lb, 99),
                                batches=sb["batches"], max_batch=sb["max_batch_graphs"]))
        if gp is not None:
            row["per_graph"] = dict(graphs_per_s=gp, p50_ms=pct(lp, 50), p99_ms=pct(lp, 99))
        else:
            row["per_graph"] = "not run: arrival rate above 1.5x its saturation (queue grows without bound)"
        rates.append(row)
    # whole job: every rank serves its own stream; throughput adds up, the
    # latency percentiles are the worst rank's
    _, sat_b_all, (p50_b, p99_b) = reduce_over_ranks(world, dev, 0.0, sat_b, (pct(lat_b, 50), pct(lat_b, 99)))
    _, sat_p_all, (p50_p, p99_p) = reduce_over_ranks(world, dev, 0.0, sat_p, (pct(lat_p, 50), pct(lat_p, 99)))
    out = dict(
        metric=METRIC, value=sat_b_all, unit="graphs/s", n_gpus=world, steps=nreq, warmup=nreq,
        ms_per_step=1e3 / sat_b, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="u64", data="synthetic",
        config=dict(workload=WORKLOADS["serve_poisson"], requests_per_rate=nreq, pool=len(pool),
                    large_graphs=len(large), generation_s=gen_s,
                    step="one request: H2D of its CSR, prepare + count in a batch, D2H of its total"),
        saturation=dict(batched=dict(graphs_per_s=sat_b_all, p50_ms=p50_b, p99_ms=p99_b,
                                     batches=st_b["batches"], max_batch=st_b["max_batch_graphs"],
                                     peak_bytes=st_b["peak_bytes_in_use"]),
                        per_graph=dict(graphs_per_s=sat_p_all, p50_ms=p50_p, p99_ms=p99_p)),
        rates=rates)
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist_done(world)
    return 0


def algorithmic_bytes(W: int, m: int, n: int, outputs: str = "total") -> int:
    """Bytes the count must move at least once: 4 B per processed wedge (the
    end id), 12 B per oriented edge (middle id + the middle's offset), 12 B
    per start (offset + cut).  With per-vertex and per-edge outputs, the
    second walk reads the same again (ends, middles, starts); the per-edge
    sums live in one uint64 per G* slot (2m of them), written once when
    cleared and read once when the two slots of each edge are combined,
    which also reads both slots' edge ids (4 B each); the outputs are
    written once (8 B per edge and per vertex)."""
    B = 4 * W + 12 * m + 12 * n
    if outputs == "all":
        B += (4 * W + 12 * m + 12 * n) + 2 * 16 * m + 8 * m + 8 * m + 8 * n
    return B


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured")
    return dict(hbm_gbs=6800.0, source="fallback")


def count_kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("count.cu", "bfc_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1812_00283_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(workload: str, outputs: str = "total", orientation: int = 0):
    """DRAM bytes per count launch from a committed ncu summary, if it was
    taken on this workload, outputs and orientation (Algorithm 2 or 3) with
    the current kernel source (or scaled from a smaller case of the same
    kernel, as the entry says); else None."""
    p = os.path.join(ROOT, "profiles", "count_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    for e in d.get("entries", []):
        if (e.get("source_sha256") == count_kernel_hash() and e.get("workload") == workload
                and e.get("outputs", "total") == outputs and e.get("orientation", 0) == orientation):
            return int(e["dram_bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_id: str):
        self.device_id = device_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.device_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(self.NAMES, parts[3:7]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(smax) if smax else None, reasons=sorted(reasons),
                    samples=len(sm))


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, device) -> None:
    """One process per GPU: NCCL process group (rendezvous from the env)."""
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl", device_id=device)


def dist_barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_over_ranks(world: int, device, t_max: float, units: float, extra_max=()):
    """Whole-job figures over the replicas: the slowest rank's time (max), the
    units all ranks processed (sum), and any further values taken as the
    maximum over ranks (e.g. latency percentiles).  One rank: unchanged."""
    if world <= 1:
        return t_max, units, list(extra_max)
    import torch
    import torch.distributed as dist
    mx = torch.tensor([t_max, *extra_max], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    vals = mx.cpu().tolist()
    return vals[0], float(sm.item()), vals[1:]


def dist_done(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


def default_outputs(workload: str) -> str:
    # the shopping workload is specified with per-vertex and per-edge counts
    return "all" if workload == "shopping_300m" else "total"


def oracle_run(g, outputs: str, threads: int) -> tuple[dict, float]:
    import oracle
    t0 = time.perf_counter()
    r = oracle.vp(g, threads=threads, vertices=outputs == "all", edges=outputs == "all")
    return r, time.perf_counter() - t0


def graph_stats(g) -> dict:
    """Degree statistics recorded with every single-graph result: maximum
    degrees, Σ deg² per layer and TC_new = Σ over edges of min(deg u, deg v)
    (the cost bound of Lemma 3)."""
    import numpy as np
    du = np.diff(g.off_u.astype(np.int64))
    dl = np.bincount(g.adj_u, minlength=g.num_l).astype(np.int64)
    ue = np.repeat(du, du)
    return dict(max_deg_u=int(du.max(initial=0)), max_deg_l=int(dl.max(initial=0)),
                sum_deg2_u=int((du * du).sum()), sum_deg2_l=int((dl * dl).sum()),
                tc_new=int(np.minimum(ue, dl[g.adj_u]).sum()))


def oracle_sample(g, outputs: str, threads: int, target_s: float):
    """A bounded sample of the workload for the CPU oracle: the subgraph of a
    seeded fraction of U (the whole graph when that fraction reaches 1),
    sized from a calibration run on a small sample so that one run takes
    about target_s.  Returns (graph, fraction, one run's result, seconds)."""
    from bfc_inputs import generators as G

    def sample(f):
        return g if f >= 1.0 else G.sample_u(g, f, 77)
    f = min(1.0, 1e6 * max(threads, 1) / max(g.num_edges, 1))
    s = sample(f)
    r, dt = oracle_run(s, outputs, threads)
    nf = min(1.0, f * target_s / max(dt, 1e-3))
    if nf <= f:
        return s, f, r, dt
    s = sample(nf)
    r, dt = oracle_run(s, outputs, threads)
    return s, nf, r, dt


def sample_desc(workload: str, frac: float, sample, r: dict, outputs: str) -> str:
    what = f"full {workload} graph" if frac == 1.0 else \
        f"{workload} graph restricted to a seeded {100 * frac:.3g}% of U"
    outs = "total + per-vertex + per-edge" if outputs == "all" else "total"
    return f"{what}, {sample.num_edges} edges, W={r['wedges']}, {outs}; oracle incl. its own preparation"


def run_reference(args, rank, world):
    """The CPU oracle (Algorithm 2 scheduled as Algorithm 5) timed on the
    host cores, on the same workload (a bounded sample of it)."""
    if rank != 0:
        return 0
    args.workload = args.workload or HEADLINE
    # the inputs are drawn on the GPU when there is one (the same graph as the
    # numpy generator's, in seconds instead of minutes for the 300M-edge
    # workload); only the oracle is timed, on the host cores
    gen_dev = "cpu"
    try:
        import torch
        if torch.cuda.is_available():
            gen_dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    except ImportError:
        pass
    g = make_graph(args.workload, 0, gen_dev)
    outputs = args.outputs or default_outputs(args.workload)
    threads = os.cpu_count() or 1
    per_step = min(10.0, 150.0 / (args.steps + args.warmup))
    sample, frac, r, _ = oracle_sample(g, outputs, threads, per_step)
    times, W = [], r["wedges"]
    for i in range(args.warmup + args.steps):
        r, dt = oracle_run(sample, outputs, threads)
        if i >= args.warmup:
            times.append(dt)
    v = W * len(times) / sum(times)
    desc = sample_desc(args.workload, frac, sample, r, outputs) + "; timed per step"
    out = dict(metric=METRIC, value=v, unit=UNIT, impl="reference", n_gpus=world,
               steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * statistics.mean(times),
               higher_is_better=True, scaling="weak", vs_baseline=None, dtype="u64",
               data="synthetic", config=dict(workload=WORKLOADS[args.workload]),
               cpu_baseline=dict(value=v, unit=UNIT, cores=threads, kind="oracle", sample=desc),
               e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help=f"default: {HEADLINE} (total + per-vertex + per-edge) with the 20M-edge "
                         "power-law total count under its own key")
    ap.add_argument("--no-history", action="store_true",
                    help="default workload only, without the 20M-edge power-law line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--orientation", type=int, default=0, choices=[0, 1],
                    help="0 = Algorithm 2 (start highest), 1 = Algorithm 3 (end highest)")
    ap.add_argument("--outputs", default=None, choices=["total", "all"],
                    help="total only, or total + per-vertex + per-edge (default: all for shopping_300m)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--core-vertices", type=int, default=None,
                    help="total counts: the top-K priority core counted by the tensor-core product "
                         "(default: the library's automatic choice)")
    ap.add_argument("--sparsify-samples", type=int, default=16,
                    help="approximate counting on the 20M-edge power-law graph: samples per estimate "
                         "(0 = skip)")
    ap.add_argument("--sparsify-p", type=float, nargs="+", default=[0.1, 0.05, 0.2],
                    help="keep probabilities of the approximate-counting runs (the first is checked "
                         "against the oracle)")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--serve-pool", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[0.25, 0.5, 1.0, 1.5],
                    help="arrival rates as fractions of the batched server's saturation")
    ap.add_argument("--serve-rates-per-graph", type=float, nargs="*", default=[0.5, 0.9],
                    help="arrival rates as fractions of the per-graph server's saturation")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch_4096":
        return run_batch(args, rank, world)
    if args.workload == "serve_poisson":
        return run_serve(args, rank, world)

    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, dev)
    workload = args.workload or HEADLINE
    outputs = args.outputs or default_outputs(workload)
    out = run_single(args, workload, outputs, rank, world, local, dev)
    if args.workload is None and not args.no_history:
        # the 20M-edge power-law graph, total count only: the count kernel's
        # history is quoted on this workload
        h = run_single(args, "powerlaw_20m", "total", rank, world, local, dev, one_thread=False)
        out["powerlaw_20m"] = {k: h[k] for k in ("value", "unit", "ms_per_step", "roofline", "e2e",
                                                 "cpu_baseline", "gpu_launches", "clocks")}
        out["powerlaw_20m"]["config"] = {k: h["config"][k] for k in (
            "workload", "wedges_per_step", "butterflies", "prepare_ms_median", "count_ms_median",
            "count_only_wedges_per_s", "outputs", "oracle_agrees")}
        if args.sparsify_samples > 0:
            out["sparsified"] = run_sparsified(args, rank, dev, int(h["config"]["butterflies"]))
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist_done(world)
    return 0


def run_sparsified(args, rank: int, dev, exact: int, seed: int = 7) -> dict:
    """Section 7's estimator with this counter as its inner block, on the
    20M-edge power-law graph: args.sparsify_samples edge-sparsified copies
    (each edge kept with probability p) sampled, prepared and counted as one
    batch, then the estimate, per call of bfc_estimate_sparsified (inputs
    resident, L2 flushed between calls); the count launch of the prepared
    samples timed alone for its roofline."""
    import torch

    from paper_1812_00283_gb300 import bfc

    g = make_graph("powerlaw_20m", rank, dev)
    off = torch.from_numpy(g.off_u).to(dev)
    adj = torch.from_numpy(g.adj_u).to(dev)
    r, l, m = g.num_u, g.num_l, g.num_edges
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    k = args.sparsify_samples
    counts = torch.zeros(k, dtype=torch.int64, device=dev)
    est = torch.zeros(2, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peaks = measured_peaks()
    steps = max(1, min(args.steps, 5))
    runs = []
    for p in args.sparsify_p:
        def call(ev=None):
            if ev:
                ev[0].record(stream)
            bfc.bfc_estimate_sparsified(r, l, m, off.data_ptr(), adj.data_ptr(), p, seed, k, None, sp,
                                        counts.data_ptr(), est.data_ptr())
            if ev:
                ev[1].record(stream)
        for _ in range(args.warmup):
            flush.fill_(1)
            call()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 0xff)
            call(evs[i])
        torch.cuda.synchronize()
        ms = statistics.median(e[0].elapsed_time(e[1]) for e in evs)
        e, se = est.cpu().tolist()
        # the count launch over the prepared samples, alone
        h = bfc.bfc_prepare_sparsified(r, l, m, off.data_ptr(), adj.data_ptr(), p, seed, k, None, sp)
        info = bfc.bfc_graph_info(h)
        tot2 = torch.zeros(k, dtype=torch.int64, device=dev)
        bfc.bfc_count_batch(h, sp, tot2.data_ptr())
        cev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3)]
        for c in cev:
            flush.fill_(2)
            c[0].record(stream)
            bfc.bfc_count_batch(h, sp, tot2.data_ptr())
            c[1].record(stream)
        bfc.bfc_sync(h, sp)
        bfc.bfc_release(h)
        if not torch.equal(tot2, counts):
            raise SystemExit("sampled counts differ between the one-call and the prepared path")
        if not runs:
            first = counts.clone()
        cnt_ms = statistics.median(c[0].elapsed_time(c[1]) for c in cev)
        Ws, ms_, ns = int(info["wedges"]), int(info["num_edges"]), int(info["num_u"]) + int(info["num_l"])
        B = algorithmic_bytes(Ws, ms_, ns, "total")
        runs.append(dict(p=p, samples=k, ms_per_estimate=ms, samples_per_s=k / (ms / 1e3),
                         sampled_wedges_per_s=Ws / (ms / 1e3), sampled_edges=ms_, sampled_wedges=Ws,
                         estimate=e, std_error=se, rel_error=(e - exact) / exact if exact else None,
                         count_ms=cnt_ms,
                         count_roofline=dict(bound="hbm", achieved=B / (cnt_ms / 1e3) / 1e9,
                                             peak=peaks["hbm_gbs"], unit="GB/s",
                                             frac=B / (cnt_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                                             kernel="k_count (bfc_count_batch over the samples)",
                                             algorithmic_bytes_per_launch=B)))
    out = dict(workload="powerlaw_20m", exact=exact, seed=seed, runs=runs,
               note="bfc_estimate_sparsified: sampling (SplitMix64 per sample and edge), prepare of "
                    "the samples as one batch, one count launch, estimate; median of "
                    f"{steps} calls after {args.warmup} warm-up calls, L2 flushed between calls")
    if rank == 0 and not args.no_cpu_baseline and runs:
        import oracle
        p = args.sparsify_p[0]
        t0 = time.perf_counter()
        ref = oracle.vp(oracle.sparsify(g, p, seed, 0), threads=os.cpu_count() or 1)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = dict(value=1e3 * dt, unit="ms per sample", cores=os.cpu_count() or 1,
                                   kind="oracle", sample=f"sample 0 of p={p}: oracle sparsify + Algorithm 2")
        out["oracle_agrees"] = ref["total"] == int(first.cpu().numpy().view("uint64")[0])
    return out


def run_single(args, workload: str, outputs: str, rank: int, world: int, local: int, dev,
               one_thread: bool = True) -> dict:
    """One graph, prepared and counted per step (the single-graph hot path):
    the bench line of that workload, with its roofline, CPU baseline and
    end-to-end figures."""
    import torch

    from paper_1812_00283_gb300 import bfc

    g = make_graph(workload, rank, dev)
    off = torch.from_numpy(g.off_u).to(dev)
    adj = torch.from_numpy(g.adj_u).to(dev)
    r, l, m = g.num_u, g.num_l, g.num_edges
    n = r + l
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    step_opts = bfc.bfc_options_init(orientation=args.orientation)
    if args.core_vertices is not None:
        step_opts.core_vertices = args.core_vertices
    if outputs == "all":
        per_u = torch.empty(max(r, 1), dtype=torch.int64, device=dev)
        per_l = torch.empty(max(l, 1), dtype=torch.int64, device=dev)
        per_e = torch.empty(max(m, 1), dtype=torch.int64, device=dev)

    def one_step(ev=None):
        if ev:
            ev[0].record(stream)
        h = bfc.bfc_prepare(r, l, m, off.data_ptr(), adj.data_ptr(), step_opts, sp)
        if ev:
            ev[1].record(stream)
        if outputs == "all":
            bfc.bfc_count_all(h, sp, per_u.data_ptr(), per_l.data_ptr(), per_e.data_ptr(), total.data_ptr())
        else:
            bfc.bfc_count(h, sp, total.data_ptr())
        if ev:
            ev[2].record(stream)
        info = bfc.bfc_graph_info(h)
        bfc.bfc_release(h)
        if ev:
            ev[3].record(stream)
        return info

    info = None
    for _ in range(args.warmup):
        flush.fill_(1)
        info = one_step()
    torch.cuda.synchronize()
    expect = int(total.item()) & ((1 << 64) - 1)
    W = int(info["wedges"])

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    props = torch.cuda.get_device_properties(dev)
    clk = ClockSampler(f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local))
    dist_barrier(world)
    torch.cuda.synchronize()
    launches0 = bfc.bfc_kernel_launches()
    clk.start()
    for i in range(args.steps):
        flush.fill_(i & 0xff)          # L2 flush between steps, outside the events
        one_step(evs[i])
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = bfc.bfc_kernel_launches() - launches0
    dist_barrier(world)
    got = int(total.item()) & ((1 << 64) - 1)
    if got != expect:
        raise SystemExit(f"count changed between steps: {got} vs {expect}")

    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    prep_ms = [e[0].elapsed_time(e[1]) for e in evs]
    count_ms = [e[1].elapsed_time(e[2]) for e in evs]
    t_total, W_all, _ = reduce_over_ranks(world, dev, sum(step_ms), W)
    value = W_all * args.steps / (t_total / 1e3)

    peaks = measured_peaks()
    cnt_s = statistics.median(count_ms) / 1e3
    B = algorithmic_bytes(W, m, n, outputs)
    achieved = B / cnt_s / 1e9
    traffic = recorded_traffic(workload, outputs, args.orientation)
    roofline = dict(bound="hbm", achieved=achieved, peak=peaks["hbm_gbs"], unit="GB/s",
                    frac=achieved / peaks["hbm_gbs"], traffic=traffic,
                    kernel="k_count (bfc_count_all)" if outputs == "all" else "k_count (bfc_count)",
                    peak_source=peaks["source"],
                    algorithmic_bytes_per_launch=B, count_ms_median=1e3 * cnt_s)

    # derived statistic (Section 1): caterpillars and the bipartite clustering
    # coefficient 4·⋈ / caterpillars, on a prepared graph (outside the steps)
    hd = bfc.bfc_prepare(r, l, m, off.data_ptr(), adj.data_ptr(), step_opts, sp)
    cat_t = torch.zeros(1, dtype=torch.int64, device=dev)
    coef_t = torch.zeros(1, dtype=torch.float64, device=dev)
    bfc.bfc_caterpillars(hd, sp, cat_t.data_ptr())     # warm-up
    ce0, ce1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ce0.record(stream)
    bfc.bfc_caterpillars(hd, sp, cat_t.data_ptr())
    ce1.record(stream)
    # total (from the timed steps, still on the device) -> coefficient, in the library
    bfc.bfc_clustering_coefficient(hd, sp, total.data_ptr(), cat_t.data_ptr(), coef_t.data_ptr())
    bfc.bfc_sync(hd, sp)
    bfc.bfc_release(hd)
    cat = int(cat_t.item()) & ((1 << 64) - 1)
    derived = dict(caterpillars=cat, clustering_coefficient=float(coef_t.item()),
                   caterpillars_ms=ce0.elapsed_time(ce1))

    # the second ceiling: one shared-memory counter increment per wedge
    # (first walk; the combined pass reads each counter again in its second)
    smem_rate, _ = bfc.bfc_bench_smem_atomics(sp, 16384)
    smem = dict(bound="smem_atomics", achieved=W / cnt_s, peak=smem_rate, unit="increments/s",
                frac=(W / cnt_s) / smem_rate,
                note="peak = bfc_bench_smem_atomics (returning 32-bit shared atomicAdd on packed "
                     "16-bit counters at random indexes, one 1024-thread CTA per SM), measured in this run")

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if args.e2e_steps > 0 and outputs == "all":
        # through the C ABI from and to page-locked host buffers:
        # bfc_count_all_host copies the CSR in, prepares, counts with all
        # outputs and copies the per-vertex, per-edge arrays and the total out
        off_h = torch.from_numpy(g.off_u).pin_memory()
        adj_h = torch.from_numpy(g.adj_u).pin_memory()
        pu_h = torch.empty(max(r, 1), dtype=torch.int64).pin_memory()
        pl_h = torch.empty(max(l, 1), dtype=torch.int64).pin_memory()
        pe_h = torch.empty(max(m, 1), dtype=torch.int64).pin_memory()
        ts = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tot, wd = bfc.bfc_count_all_host(r, l, m, off_h.data_ptr(), adj_h.data_ptr(), step_opts, sp,
                                             pu_h.data_ptr(), pl_h.data_ptr(), pe_h.data_ptr())
            ts.append(time.perf_counter() - t0)
            if tot != expect or wd != W:
                raise SystemExit("end-to-end count disagrees with the device-resident count")
        if not torch.equal(pe_h[:m], per_e[:m].cpu()):
            raise SystemExit("end-to-end per-edge counts disagree with the device-resident pass")
        ts = ts[1:]
        e2e = dict(value=W / statistics.median(ts), unit=UNIT,
                   h2d_bytes_per_step=4 * (r + 1) + 4 * m, d2h_bytes_per_step=8 * (r + l + m) + 8,
                   ms_per_step=1e3 * statistics.median(ts),
                   note="bfc_count_all_host from page-locked host buffers: H2D of the CSR, prepare, "
                        "count with all outputs, D2H of per-vertex, per-edge and total")
    elif args.e2e_steps > 0:
        off_h = torch.from_numpy(g.off_u).pin_memory()
        adj_h = torch.from_numpy(g.adj_u).pin_memory()
        ts = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tot, wd = bfc.bfc_count_host(r, l, m, off_h.data_ptr(), adj_h.data_ptr(), step_opts, sp)
            ts.append(time.perf_counter() - t0)
            if tot != expect or wd != W:
                raise SystemExit("end-to-end count disagrees with the device-resident count")
        ts = ts[1:]
        e2e = dict(value=W / statistics.median(ts), unit=UNIT,
                   h2d_bytes_per_step=4 * (r + 1) + 4 * m, d2h_bytes_per_step=8,
                   ms_per_step=1e3 * statistics.median(ts),
                   note="bfc_count_host: H2D of the CSR, prepare, count, D2H of the total")

    cpu = None
    verified = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        sample, frac, ref, dt = oracle_sample(g, outputs, threads, 15.0)
        if frac == 1.0:
            verified = (ref["total"] == expect and ref["wedges"] == W)
        cpu = dict(value=ref["wedges"] / dt, unit=UNIT, cores=threads, kind="oracle",
                   sample=sample_desc(workload, frac, sample, ref, outputs) + f", one run, {dt:.1f} s")
        if one_thread:
            # the same oracle on one core, on a smaller sample (~10 s)
            s1, f1, r1, dt1 = oracle_sample(g, outputs, 1, 10.0)
            cpu["one_thread"] = dict(value=r1["wedges"] / dt1, unit=UNIT, cores=1,
                                     sample=sample_desc(workload, f1, s1, r1, outputs) +
                                     f", one run, {dt1:.1f} s")

    out = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=t_total / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="u64", data="synthetic",
        config=dict(workload=WORKLOADS[workload], num_u=r, num_l=l, num_edges=m,
                    wedges_per_step=W, butterflies=expect, graph=graph_stats(g), derived=derived,
                    step="prepare (a1-a5) + count (a6-a7" + (", a8, a9" if outputs == "all" else "") +
                         "), CSR resident in HBM",
                    l2="flushed between steps (512 MB write outside the timed events)",
                    parallelism=f"replicas x{world} (independent graphs, no collective)",
                    orientation=["Algorithm 2 (BFC-VP)", "Algorithm 3 (BFC-VP++)"][args.orientation],
                    prepare_ms_median=statistics.median(prep_ms),
                    count_ms_median=statistics.median(count_ms),
                    count_only_wedges_per_s=W / cnt_s,
                    outputs="total + per-vertex + per-edge (bfc_count_all)" if outputs == "all"
                    else "total (bfc_count)",
                    bins=dict(dense_starts=info["dense_starts"], dense_items=info["dense_items"],
                              hash_starts=info["hash_starts"], team_starts=info["team_starts"],
                              warp_starts=info["warp_starts"]),
                    dense_core=dict(vertices_u=info["core_u"], vertices_l=info["core_l"],
                                    used_by=("bfc_count (total)" if info["core_u"] + info["core_l"] and
                                             outputs == "total" else "not used")),
                    oracle_agrees=verified),
        roofline=roofline, smem_roofline=smem, cpu_baseline=cpu, e2e=e2e,
        gpu_launches=launches, clocks=clocks)
    del off, adj
    if outputs == "all":
        del per_u, per_l, per_e
    torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    sys.exit(main())
