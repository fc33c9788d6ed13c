"""Runs a few time steps of a named workload with the step's kernels launched
one by one, for kernel profilers (ncu cannot see kernels inside CUDA graphs
that contain conditional nodes, which is how the library normally runs).

    python -m paper_2104_11404_gb300.profile_step --workload tg2d_64 --precision mixed --steps 5
"""
import argparse
import json
import os
import sys


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="tg2d_64")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--graph", action="store_true", help="keep the CUDA graph launches")
    args = ap.parse_args()
    import torch

    from . import build as libbuild
    from . import workloads as W
    from .hydro import Hydro
    libbuild.build()
    torch.cuda.set_device(0)
    cfg = W.CONFIGS[args.workload]
    g = Hydro(cfg, precision=args.precision,
              phys_overrides=None if args.graph else {"direct_launch": 1})
    g.init_state()
    if args.warmup:
        g.run_to(cfg["t_final"], max_steps=args.warmup)
    st = g.run_to(cfg["t_final"], max_steps=args.steps)
    print(json.dumps({"workload": args.workload, "precision": args.precision, **st}))
    g.close()


if __name__ == "__main__":
    sys.exit(main())
