"""Enumerate one of the seeded synthetic workloads on the current GPU.

    python -m paper_2401_05039_gb300 chunglu20k [--repeat 3] [--schedule 0] [--steal 1]
                                                [--layout 0] [--blocks-per-sm 0] [--prune 0]

Prints count, hash, nodes, algorithmic bytes, device milliseconds and the
device memory the library holds after the first run, one line per repeat.
This is the fixed command the kernel profiles are taken on.
"""
from __future__ import annotations

import argparse
import os
import sys


def main() -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2401_05039_gb300")
    ap.add_argument("workload", help="er200x300 | chunglu20k | planted5k | chunglu200k | batchgraph:<i> (graph i "
                                     "of the 4,096-graph batch)")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--schedule", type=int, default=0)
    ap.add_argument("--steal", type=int, default=1)
    ap.add_argument("--layout", type=int, default=0, help="0 auto, 1 rows, 2 columns")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="0 = default (2 blocks of 256 threads)")
    ap.add_argument("--prune", type=int, default=0, help="1 = iMBE's L - L' removal (column layout)")
    args = ap.parse_args()

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import synth

    from . import mbe

    mbe.load()
    if args.workload.startswith("batchgraph:"):
        g = synth.batch_graph(3 + int(args.workload.split(":", 1)[1]))
    else:
        g = synth.workload(args.workload)
    G = mbe.Graph.from_synth(g)
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(args.repeat):
        r = G.enumerate(schedule=args.schedule, steal=args.steal, layout=args.layout,
                        blocks_per_sm=args.blocks_per_sm, prune=args.prune)
        torch.cuda.synchronize()
        held = (free0 - torch.cuda.mem_get_info()[0]) / 2**30
        print(f"{args.workload} run {k}: count {r.count} hash {r.hash:#018x} nodes {r.nodes} bytes_alg {r.bytes_alg} "
              f"device_ms {r.device_ms:.3f} workers {r.n_workers} workspace_gib {held:.2f}", flush=True)
    G.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
