"""Runs a few time steps of a named workload with the step's kernels launched
one by one, for kernel profilers (ncu cannot see kernels inside CUDA graphs
that contain conditional nodes, which is how the library normally runs).

    python -m paper_2104_11404_gb300.profile_step --workload tg2d_64 --precision mixed --steps 5
    python -m paper_2104_11404_gb300.profile_step --batch --steps 2 --tuning 1024,1,1

--rom runs the reduced model of the 3D blast 8^3 (offline: snapshots and POD;
then online hyper-reduced steps).
--batch runs the 512-instance point-blast sweep through the batched form
instead (its attempt graph holds kernel nodes only, so profilers see them);
--tuning threads,ctas_per_sm,smem_lines[,qpt] fixes the launch shape (no autotuner
launches before the profiled ones).  --apply N instead applies the CG
preconditioner N times to a random vector (the plain band passes, as bench.py
times them for its roofline line).
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
    ap.add_argument("--batch", action="store_true", help="the batched point-blast sweep")
    ap.add_argument("--instances", type=int, default=512)
    ap.add_argument("--tuning", default="", help="threads,ctas_per_sm,smem_lines[,qpt]")
    ap.add_argument("--precond", type=int, default=-1,
                    help="cg_precond (0 Jacobi, 1 tensor bands, 2 exact); default: the library's")
    ap.add_argument("--apply", type=int, default=0,
                    help="apply the CG preconditioner this many times instead of stepping")
    ap.add_argument("--rom", action="store_true",
                    help="the reduced model of the 3D blast 8^3 (snapshots, POD, online steps)")
    args = ap.parse_args()
    if args.batch:
        return run_batch(args)
    if args.rom:
        return run_rom(args)
    import torch

    from . import build as libbuild
    from . import workloads as W
    from .hydro import Hydro
    libbuild.build()
    torch.cuda.set_device(0)
    cfg = W.CONFIGS[args.workload]
    over = {} if args.graph else {"direct_launch": 1}
    if args.precond >= 0:
        over["cg_precond"] = args.precond
    g = Hydro(cfg, precision=args.precision, phys_overrides=over or None)
    g.init_state()
    if args.apply:
        from . import lagh
        nv = g.get_state()[0].numel()
        gen = torch.Generator(device="cuda").manual_seed(0)
        r = torch.randn(nv, dtype=torch.float64, device="cuda", generator=gen)
        z = torch.empty_like(r)
        for _ in range(args.apply):
            lagh.lh_precond_apply(g.ctx, r, z)
        torch.cuda.synchronize()
        print(json.dumps({"workload": args.workload, "applied": args.apply,
                          "z_norm": float(z.norm())}))
        g.close()
        return 0
    if args.warmup:
        g.run_to(cfg["t_final"], max_steps=args.warmup)
    st = g.run_to(cfg["t_final"], max_steps=args.steps)
    print(json.dumps({"workload": args.workload, "precision": args.precision, **st}))
    g.close()


def run_batch(args):
    import torch

    from . import build as libbuild
    from . import workloads as W
    from .batch import Batch
    libbuild.build()
    torch.cuda.set_device(0)
    tuning = None
    if args.tuning:
        f = [int(v) for v in args.tuning.split(",")]
        tuning = dict(threads=f[0], ctas_per_sm=f[1], smem_lines=f[2], qpt=f[3] if len(f) > 3 else 1)
    b = Batch(W.batch_instances(args.instances), precision=args.precision, tuning=tuning)
    b.init_state()
    if tuning is None:
        b.autotune()
    if args.warmup:
        b.run_to(0.8, max_steps=args.warmup)
    st = b.run_to(0.8, max_steps=args.steps)
    print(json.dumps({"batch": args.instances, "precision": args.precision, "tuning": b.tuning(),
                      **st}))
    b.close()


def run_rom(args):
    """Offline stage (batched FP64 run with snapshot capture, POD of each field)
    and then --steps online steps of the hyper-reduced model (after --warmup),
    on the 3D blast 8^3 Q2/Q1 over t in [0, 0.1]."""
    import torch

    from . import build as libbuild
    from . import lagh
    from . import workloads as W
    from .batch import Batch
    from .hydro import Hydro
    from .rom import Rom
    libbuild.build()
    torch.cuda.set_device(0)
    cfg = W.scaled("sedov3d_32", n=(8, 8, 8), t_final=0.1)
    b = Batch([cfg], precision="fp64")
    b.init_state()
    v0, e0, x0 = (a.clone() for a in b.get_state())
    Sv, Se, Sx = b.snapshots([0], 8000)
    b.run_to(0.1)
    (_, cnt, V, E, X), = b.snapshot_views(Sv, Se, Sx)
    bases, sweeps = [], []
    for cols, off in ((V, v0), (E, e0), (X, x0)):
        n, m = cols.shape
        U = torch.zeros(n * m, dtype=torch.float64, device="cuda")
        sig = torch.zeros(n, dtype=torch.float64, device="cuda")
        work = torch.zeros(m * n + 2 * n + 16, dtype=torch.float64, device="cuda")
        k, sw = lagh.lh_pod(cols.contiguous(), m, n, off, 0.9999, U, sig, work,
                            torch.cuda.current_stream().cuda_stream)
        bases.append(U.view(n, m)[:k].contiguous())
        sweeps.append(sw)
    b.close()
    g = Hydro(cfg, precision="fp64")
    nb = [B.shape[0] for B in bases]
    r = Rom(g, bases[0], bases[1], bases[2], v0, e0, x0, 2 * nb[0], 2 * nb[1])
    if args.warmup:
        r.run_to(0.1, max_steps=args.warmup)
    st = r.run_to(0.1, max_steps=args.steps)
    print(json.dumps({"rom": "sedov3d_8", "snapshots": cnt, "basis": nb, "pod_sweeps": sweeps,
                      "sampled_elements": int(r.info.n_elems), **st}))
    r.close()
    g.close()


if __name__ == "__main__":
    sys.exit(main())
