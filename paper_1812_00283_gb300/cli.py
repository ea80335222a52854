"""Command-line butterfly counter for the synthetic workloads.

    python -m paper_1812_00283_gb300.cli --workload powerlaw_20m --repeat 2 --mode total

Generates the seeded workload on the GPU, prepares it once and runs the
requested count `repeat` times, printing the result and per-call device
times (CUDA events on the launching stream).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def workload(name: str, device):
    from bfc_inputs import generators as G
    table = {
        "uniform_small": lambda: G.uniform_small(device=device),
        "powerlaw_20m": lambda: G.powerlaw_20m(device=device),
        "shopping_300m": lambda: G.shopping_300m(device=device),
        "shopping_30m": lambda: G.shopping_300m(device=device, scale=0.1),
        "shopping_3m": lambda: G.shopping_300m(device=device, scale=0.01),
    }
    if name not in table:
        raise SystemExit(f"unknown workload {name}; choose from {sorted(table)}")
    return table[name]()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="powerlaw_20m")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--mode", default="total", choices=["total", "vertices", "edges", "all"])
    ap.add_argument("--warp-max-work", type=int, default=None)
    ap.add_argument("--hash-max-work", type=int, default=None)
    ap.add_argument("--team-max-work", type=int, default=None)
    ap.add_argument("--orientation", type=int, default=0, choices=[0, 1])
    ap.add_argument("--core-vertices", type=int, default=-1,
                    help="top-K priority core counted by the tensor-core product (total counts)")
    args = ap.parse_args(argv)

    import torch

    from paper_1812_00283_gb300 import bfc

    dev = torch.device("cuda", 0)
    g = workload(args.workload, dev)
    off = torch.from_numpy(g.off_u).to(dev)
    adj = torch.from_numpy(g.adj_u).to(dev)
    opts = bfc.bfc_options_init()
    if args.warp_max_work is not None:
        opts.warp_max_work = args.warp_max_work
    if args.hash_max_work is not None:
        opts.hash_max_work = args.hash_max_work
    if args.team_max_work is not None:
        opts.team_max_work = args.team_max_work
    opts.orientation = args.orientation
    opts.core_vertices = args.core_vertices
    s = torch.cuda.current_stream()
    sp = s.cuda_stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    h = bfc.bfc_prepare(g.num_u, g.num_l, g.num_edges, off.data_ptr(), adj.data_ptr(), opts, sp)
    e1.record(s)
    torch.cuda.synchronize()
    prep_ms = e0.elapsed_time(e1)
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    pu = torch.empty(max(g.num_u, 1), dtype=torch.int64, device=dev)
    pl = torch.empty(max(g.num_l, 1), dtype=torch.int64, device=dev)
    pe = torch.empty(max(g.num_edges, 1), dtype=torch.int64, device=dev)
    times = []
    for _ in range(args.repeat):
        e0.record(s)
        if args.mode == "total":
            bfc.bfc_count(h, sp, total.data_ptr())
        elif args.mode == "vertices":
            bfc.bfc_count_vertices(h, sp, pu.data_ptr(), pl.data_ptr(), total.data_ptr())
        elif args.mode == "edges":
            bfc.bfc_count_edges(h, sp, pe.data_ptr(), total.data_ptr())
        else:
            bfc.bfc_count_all(h, sp, pu.data_ptr(), pl.data_ptr(), pe.data_ptr(), total.data_ptr())
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    bfc.bfc_sync(h, sp)
    info = bfc.bfc_graph_info(h)
    bfc.bfc_release(h)
    print(json.dumps(dict(workload=g.name, mode=args.mode, butterflies=int(total.item()) & ((1 << 64) - 1),
                          wedges=info["wedges"], prepare_ms=prep_ms, count_ms=times, info=info)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
