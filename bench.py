"""Benchmark: Lagrangian step DOF-updates/s of the full-order hydro step.

Workload: the 2D Taylor-Green vortex of Section 6.1.3 on 64x64 Q2/Q1 elements
(the workload the headline metric is quoted on), synthetic (problem initial
conditions, no data).  One bench step = CHUNK accepted RK2-average time steps
of the device-controlled time loop (lh_run_to).  value = (2 N_V + N_E) x
accepted time steps / device time, for the mixed FP32/FP64 path; the FP64 path
is measured the same way and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
Under torchrun every rank advances its own instance (independent replicas,
weak scaling, no collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CHUNK = 50           # accepted time steps per bench step
WORKLOAD = "tg2d_64"
BATCH_CHUNK = 20     # accepted time steps of every instance per batched bench step
# DRAM read + write per launch of the preconditioner kernel on this workload,
# from an ncu capture (cold caches); None until the current kernel is captured
PASS_KERNEL_DRAM_BYTES = 437163  # cg_pass2d_kernel on tg2d_64: mean of 3 launches, 0 written


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_reduce(x, op, world, device):
    """Max ("max") or sum ("sum") of a scalar over the ranks of the process
    group, through a tensor on `device` ("cuda" with NCCL, "cpu" with gloo);
    the value itself at world size 1."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    red = torch.distributed.ReduceOp.MAX if op == "max" else torch.distributed.ReduceOp.SUM
    torch.distributed.all_reduce(t, op=red)
    return float(t.item())



class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        except Exception:
            return out
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        busy = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        out["sm_mhz"] = statistics.median(busy) if busy else None
        out["sm_max_mhz"] = max(mx) if mx else None
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


def flops_per_element_force(dim, k, mixed):
    """Algorithmic flops of one element in the force kernel: the trip counts
    of the sum-factorised contractions (2 flops per multiply-add) plus a fixed
    budget for the quadrature-point physics (300 flops per point in 2D, 600 in
    3D: Jacobian algebra, EOS, sound speed, eigen-direction viscosity, stress,
    time-step bound)."""
    P, NQ = k + 1, 2 * k
    ND1, ND2, NQD = P ** dim, k ** dim, NQ ** dim
    nf = 2 * dim                       # x and v, dim components each
    if dim == 2:
        interp = nf * P * NQ * P * 2 + NQD * nf * P * 3
    else:
        interp = nf * P * P * NQ * P * 2 + nf * P * NQ * NQ * P * 3 + NQD * nf * P * 4
    eq = NQD * ND2 * (dim)             # e at the points
    phys = NQD * (300 if dim == 2 else 600)
    if not mixed:
        if dim == 2:
            trans = dim * dim * P * NQ * NQ + dim * ND1 * dim * NQ
        else:
            trans = dim * dim * P * NQ * NQ * NQ + dim * dim * P * P * NQ * NQ + dim * ND1 * dim * NQ
    else:
        PK = P * k
        if dim == 2:
            trans = dim * dim * PK * NQ * NQ * 2 + dim * ND1 * ND2 * dim * NQ * 2
        else:
            trans = (dim * dim * PK * NQ * NQ * NQ * 2 + dim * dim * PK * PK * NQ * NQ * 2 +
                     dim * ND1 * ND2 * dim * NQ * 2)
        trans += dim * ND1 * ND2       # FP64 row sums
    return 2 * (interp + eq + trans) + phys


def _env_info():
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    return peaks


def run_native(args):
    import torch
    from paper_2104_11404_gb300 import build as libbuild
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.hydro import Hydro

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    libbuild.build()
    cfg = W.CONFIGS[WORKLOAD]
    nv, ne, nel = W.sizes(cfg)
    N = 2 * nv + ne
    stream = torch.cuda.Stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        return rank_reduce(x, "max", world, "cuda")

    def sum_over_ranks(x):
        return rank_reduce(x, "sum", world, "cuda")

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def measure(precision):
        with torch.cuda.stream(stream):
            g = Hydro(cfg, precision=precision, stream=stream,
                      phys_overrides={"direct_launch": 1} if args.direct_launch else None)
            g.init_state()
            for _ in range(args.warmup):
                g.run_to(cfg["t_final"], max_steps=CHUNK)
            torch.cuda.synchronize()
            barrier()
            torch.cuda.synchronize()
            dev_ms, steps, cg, rejects = 0.0, 0, 0, 0
            clk = Clocks(local)
            clk.start()
            t_wall = time.time()
            for _ in range(args.steps):
                flush.fill_(1.0)            # L2 flushed between timed steps
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = g.run_to(cfg["t_final"], max_steps=CHUNK)
                e1.record(stream)
                e1.synchronize()
                dev_ms += e0.elapsed_time(e1)
                steps += st["steps"]
                cg += st["cg_iters"]
                rejects += st["rejects"]
            wall = time.time() - t_wall
            clocks = clk.stop()
            torch.cuda.synchronize()
            barrier()
            # end to end through the C ABI with pinned host buffers
            hv = torch.empty(nv, dtype=torch.float64, pin_memory=True)
            he = torch.empty(ne, dtype=torch.float64, pin_memory=True)
            hx = torch.empty(nv, dtype=torch.float64, pin_memory=True)
            lagh.lh_get_state(g.ctx, hv, he, hx)
            e2e_ms, e2e_steps = 0.0, 0
            for _ in range(max(1, args.steps // 2)):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                t_, dt_ = lagh.lh_get_state(g.ctx, None, None, None)
                lagh.lh_set_state(g.ctx, hv, he, hx, t_, dt_)
                st = g.run_to(cfg["t_final"], max_steps=CHUNK)
                lagh.lh_get_state(g.ctx, hv, he, hx)
                e1.record(stream)
                e1.synchronize()
                e2e_ms += e0.elapsed_time(e1)
                e2e_steps += st["steps"]
            # dominant kernel: the force evaluation over all elements, timed
            # alone with events on the library stream
            v, e, x, _, _ = g.get_state()
            ids = torch.arange(nel, dtype=torch.int32, device="cuda")
            F1 = torch.empty(nel * cfg["dim"] * (cfg["order"] + 1) ** cfg["dim"], dtype=torch.float64,
                             device="cuda")
            lagh.lh_force_sampled(g.ctx, ids, nel, v, e, x, F1, want_dt=False)
            reps = 50
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                lagh.lh_force_sampled(g.ctx, ids, nel, v, e, x, F1, want_dt=False)
            e1.record(stream)
            e1.synchronize()
            force_ms = e0.elapsed_time(e1) / reps
            # the CG preconditioner passes (dominant by share in the launch list):
            # one application = precond_kernels launches (the tile kernel, or
            # one line pass per direction)
            r = torch.randn(nv, dtype=torch.float64, device="cuda")
            z = torch.empty_like(r)
            lagh.lh_precond_apply(g.ctx, r, z)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                lagh.lh_precond_apply(g.ctx, r, z)
            e1.record(stream)
            e1.synchronize()
            pk = g.layout.precond_kernels
            pass_ms = e0.elapsed_time(e1) / reps / pk
            g.close()
        return dict(dev_ms=max_over_ranks(dev_ms), steps=sum_over_ranks(steps), cg=cg,
                    rejects=rejects, wall=wall, clocks=clocks, e2e_ms=max_over_ranks(e2e_ms),
                    e2e_steps=sum_over_ranks(e2e_steps), force_ms=force_ms, pass_ms=pass_ms,
                    pass_kernels=pk)

    res = {p: measure(p) for p in ("mixed", "fp64")}
    batched = None if args.no_batch else measure_batched(args, stream, flush, max_over_ranks,
                                                         sum_over_ranks)
    others = None if (args.no_configs or rank != 0) else measure_configs(stream)
    if rank != 0:
        return None
    m, f = res["mixed"], res["fp64"]
    value = N * m["steps"] / (m["dev_ms"] * 1e-3)
    value64 = N * f["steps"] / (f["dev_ms"] * 1e-3)
    peaks = _env_info()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12      # TFLOP/s, unit counts x clock
    fp64_peak = 1.25                                      # TFLOP/s, GB300 nominal FP64 rate
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # one launch reads its input and writes its output (N_V doubles each): a
    # line pass along one direction, or the tile kernel's whole application
    pass_bytes = 16.0 * nv
    pass_kernel = ("cg_pass2d_kernel (CG band preconditioner, both directions on 16x16 node tiles)"
                   if m["pass_kernels"] == 1 else "cg_pass_kernel (CG band preconditioner line pass)")
    fl = flops_per_element_force(cfg["dim"], cfg["order"], True) * nel
    achieved = fl / (m["force_ms"] * 1e-3) / 1e12
    fl64 = flops_per_element_force(cfg["dim"], cfg["order"], False) * nel
    achieved64 = fl64 / (f["force_ms"] * 1e-3) / 1e12
    # kernels launched per attempt: per stage force, node gather, the initial
    # preconditioner application (pk kernels), v/x update and energy update,
    # and per CG iteration M p (element apply + node gather, one tile kernel
    # where the preconditioner is the tile kernel, pk == 1) and a
    # preconditioner application (the CG update rides on it); then control
    # and commit
    pk = m["pass_kernels"]
    per_it = (1 if pk == 1 else 2) + pk
    attempts = m["steps"] + m["rejects"]
    # every solve launches at least its kUnrolled = 3 iterations (a converged
    # solve's later ones return at once)
    launches = attempts * (2 * (4 + pk) + 2) + max(m["cg"], 3 * 2 * attempts) * per_it
    line = {
        "metric": "Lagrangian step DOF-updates/s; mixed/batched vs FP64 GPU at stated rel. error",
        "value": value,
        "unit": "DOF-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": m["dev_ms"] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "2D Taylor-Green vortex 64x64 Q2/Q1, AV on, CFL 0.1, mixed FP32/FP64",
                   "dofs_per_instance": N, "time_steps_per_bench_step": CHUNK,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "fp64": {"value": value64, "ms_per_step": f["dev_ms"] / args.steps,
                 "speedup_mixed_over_fp64": value / value64},
        "roofline": {"bound": "hbm", "kernel": pass_kernel,
                     "achieved": pass_bytes / (m["pass_ms"] * 1e-3) / 1e9, "peak": hbm_peak,
                     "unit": "GB/s", "frac": pass_bytes / (m["pass_ms"] * 1e-3) / 1e9 / hbm_peak,
                     # DRAM read + write per launch of this kernel from an ncu capture on
                     # this workload (cold caches; reset to None when the kernel changes)
                     "traffic": PASS_KERNEL_DRAM_BYTES if m["pass_kernels"] == 1 else None, "launch_us": m["pass_ms"] * 1e3,
                     "algorithmic_bytes": pass_bytes,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                     "force_kernel": {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                                      "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                                      "launch_us": m["force_ms"] * 1e3,
                                      "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock",
                                      "fp64_path": {"achieved": achieved64, "peak": fp64_peak,
                                                    "frac": achieved64 / fp64_peak,
                                                    "launch_us": f["force_ms"] * 1e3}}},
        "e2e": {"value": N * m["e2e_steps"] / (m["e2e_ms"] * 1e-3), "unit": "DOF-updates/s",
                "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8},
        "gpu_launches": int(launches),
        "clocks": m["clocks"],
    }
    if others is not None:
        line["configs"] = others
    if batched is not None:
        batched["config"] = ("512 independent 2D point-blast instances, E0 U[0.1,1], gamma "
                             "U[1.3,1.67], n x n quads with n from {16,24,32,48}, Q2/Q1, mixed, "
                             "splitmix64 seed 2104114040")
        line["batched"] = batched
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, bounded_seconds=12.0)
    return line


CONFIG_WINDOW = {"sedov2d_8": 50, "sedov3d_32": 10, "gresho2d_256": 20}


def measure_configs(stream):
    """The other workloads, each through the single-problem path in both
    precisions: a window of accepted steps from the initial state after three
    warm-up steps, device time, throughput, the mixed state's relative L2
    difference from the FP64 state after the same steps, and the mixed
    total-energy drift (the problems without an energy source)."""
    import numpy as np
    import torch
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.hydro import Hydro
    out = {}
    for name, nsteps in CONFIG_WINDOW.items():
        cfg = W.CONFIGS[name]
        res = {}
        states = {}
        for prec in ("fp64", "mixed"):
            with torch.cuda.stream(stream):
                g = Hydro(cfg, precision=prec, stream=stream)
                g.init_state()
                E0 = g.total_energy()
                g.run_to(cfg["t_final"], max_steps=3)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = g.run_to(cfg["t_final"], max_steps=nsteps)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                N = 2 * g.nv + g.ne
                v, e, x, t, _ = g.get_state()
                states[prec] = (v.cpu().numpy(), e.cpu().numpy(), t)
                res[prec] = {"value": N * st["steps"] / (ms * 1e-3), "ms_per_step": ms / st["steps"],
                             "cg_iters_per_step": st["cg_iters"] / max(1, st["steps"]),
                             "energy_drift": abs(g.total_energy() - E0) / abs(E0)}
                g.close()
        rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(a), 1e-300))
        out[name] = {"dofs": int(N), "time_steps": nsteps + 3,
                     "fp64": res["fp64"], "mixed": res["mixed"],
                     "speedup_mixed_over_fp64": res["mixed"]["value"] / res["fp64"]["value"],
                     "mixed_vs_fp64_rel_l2": {"v": rel(states["fp64"][0], states["mixed"][0]),
                                              "e": rel(states["fp64"][1], states["mixed"][1]),
                                              "t_diff": abs(states["fp64"][2] - states["mixed"][2])}}
    return out


def batch_fp64_flops(cfgs):
    """Algorithmic FP64 flops of one attempt (two stages) of the batched
    mixed step, summed over instances, with n_e elements and N_V velocity
    unknowns each (2D Q2/Q1): per element F.1 row sums 72, node gather 18,
    mass apply (two 3x3 contractions per component, scale) 234 and its gather
    18, energy update (F^T w 144, M_E^-1 32, update 4) 180; per velocity
    unknown the line solves 21 (forward and backward substitution along both
    directions, k = 2, and the scale), CG dots and updates 12, stage update 4."""
    tot = 0
    for c in cfgs:
        n = c["n"][0] * c["n"][1]
        nn = (2 * c["n"][0] + 1) * (2 * c["n"][1] + 1)
        nv = 2 * nn
        tot += 522 * n + 37 * nv
    return 2 * tot


def measure_batched(args, stream, flush, max_over_ranks, sum_over_ranks, sizes_fp64=True):
    """The 512-instance point-blast sweep (mixed), one bench step = BATCH_CHUNK
    accepted time steps of every instance (lh_batch_run_to); plus the restricted
    force on a seeded 5% element sample of every instance, and the plain
    single-problem paths on the same instance mix for the speed-up."""
    import numpy as np
    import torch
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.batch import Batch
    from paper_2104_11404_gb300.hydro import Hydro
    cfgs = W.batch_instances()
    out = {}
    with torch.cuda.stream(stream):
        b = Batch(cfgs, precision="mixed", stream=stream)
        b.init_state()
        t0 = time.time()
        tune = b.autotune(reps=2)
        tune_s = time.time() - t0
        dofs = b.dofs()
        for _ in range(args.warmup):
            b.run_to(0.8, max_steps=BATCH_CHUNK)
        torch.cuda.synchronize()
        dev_ms, dof_upd, steps, rejects, launches = 0.0, 0, 0, 0, 0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = b.run_to(0.8, max_steps=BATCH_CHUNK)
            e1.record(stream)
            e1.synchronize()
            dev_ms += e0.elapsed_time(e1)
            dof_upd += st["dof_updates"]
            steps += st["steps"]
            rejects += st["rejects"]
            launches += st["graph_launches"]
        # replicas: every rank advances its own copy of the sweep
        value = sum_over_ranks(dof_upd) / (max_over_ranks(dev_ms) * 1e-3)
        value_rank = dof_upd / (dev_ms * 1e-3)
        attempt_ms = dev_ms / max(1, launches)
        # end to end: pinned host state in, run, state out
        hv = torch.empty(b.nv, dtype=torch.float64, pin_memory=True)
        he = torch.empty(b.ne, dtype=torch.float64, pin_memory=True)
        hx = torch.empty(b.nv, dtype=torch.float64, pin_memory=True)
        lagh.lh_batch_get_state(b.b, hv, he, hx)
        q = b.query()
        e2e_ms, e2e_upd = 0.0, 0
        for _ in range(max(1, args.steps // 2)):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.set_state(hv, he, hx, q["t"], q["dt"])
            st = b.run_to(0.8, max_steps=BATCH_CHUNK)
            lagh.lh_batch_get_state(b.b, hv, he, hx)
            q = b.query()
            e1.record(stream)
            e1.synchronize()
            e2e_ms += e0.elapsed_time(e1)
            e2e_upd += st["dof_updates"]
        # restricted force on 5% of every instance's elements
        lists = [W.element_sample(c["n"][0] * c["n"][1], frac=0.05, stream=i)
                 for i, c in enumerate(cfgs)]
        nsamp = int(sum(len(l) for l in lists))
        b.force_sampled(lists)
        reps = 20
        F1, _, off, _ = b.force_sampled(lists)
        d_off = torch.from_numpy(off).to("cuda")
        d_ids = torch.from_numpy(np.concatenate(lists).astype(np.int32)).to("cuda")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            lagh.lh_batch_force_sampled(b.b, d_off, d_ids, F1)
        e1.record(stream)
        e1.synchronize()
        hr_ms = e0.elapsed_time(e1) / reps
        E_all = b.total_energy()
        b.close()
        # plain single-problem paths (one context per problem) on the same mix
        rates = {}
        if sizes_fp64:
            for prec in ("fp64", "mixed"):
                for n in W.BATCH_SIZES:
                    c = dict(cfgs[0], n=(n, n, 1), gamma=1.4, blast_energy=0.5)
                    g = Hydro(c, precision=prec, stream=stream)
                    g.init_state()
                    g.run_to(0.8, max_steps=3)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    stg = g.run_to(0.8, max_steps=BATCH_CHUNK)
                    e1.record(stream)
                    e1.synchronize()
                    N = 2 * g.nv + g.ne
                    rates[(prec, n)] = N * stg["steps"] / (e0.elapsed_time(e1) * 1e-3)
                    g.close()
    per_inst_steps = steps / len(cfgs)
    out = {"value": value, "unit": "DOF-updates/s", "instances": len(cfgs),
           "dofs_total": int(dofs.sum()), "ms_per_step": dev_ms / args.steps,
           "time_steps_per_bench_step": BATCH_CHUNK, "accepted_steps": steps, "rejects": rejects,
           "attempt_graphs": launches, "attempt_ms": attempt_ms, "tuning": tune,
           "autotune_s": tune_s,
           "e2e": {"value": e2e_upd / (e2e_ms * 1e-3), "unit": "DOF-updates/s",
                   "h2d_bytes_per_step": 8 * (2 * b.nv + b.ne) + 16 * len(cfgs),
                   "d2h_bytes_per_step": 8 * (2 * b.nv + b.ne)},
           "hyper_reduced_force": {"sampled_elements": nsamp, "launch_us": hr_ms * 1e3,
                                   "elements_per_s": nsamp / (hr_ms * 1e-3),
                                   "sample": "ceil(0.05 n_e) elements per instance, seeded "
                                             "Fisher-Yates, sorted"},
           "energy_min": float(np.min(E_all))}
    fl = batch_fp64_flops(cfgs)
    out["roofline"] = {"bound": "alu", "kernel": "batch_stage_kernel (both stages of an attempt)",
                       "achieved": fl / (attempt_ms * 1e-3) / 1e12, "peak": 1.25,
                       "unit": "TFLOP/s (FP64)",
                       "frac": fl / (attempt_ms * 1e-3) / 1e12 / 1.25,
                       "algorithmic_fp64_flops_per_attempt": fl,
                       "peak_source": "GB300 nominal FP64 rate (1.25 TFLOP/s)"}
    if rates:
        # time the same accepted steps would take through one context per problem
        def seq_time(prec):
            return sum(dofs[i] * per_inst_steps / rates[(prec, c["n"][0])] for i, c in enumerate(cfgs))
        out["single_problem_fp64"] = {"value": dofs.sum() * per_inst_steps / seq_time("fp64"),
                                      "rates_by_size": {str(n): rates[("fp64", n)] for n in W.BATCH_SIZES}}
        out["single_problem_mixed"] = {"value": dofs.sum() * per_inst_steps / seq_time("mixed"),
                                       "rates_by_size": {str(n): rates[("mixed", n)] for n in W.BATCH_SIZES}}
        out["speedup_over_fp64_single_problem"] = value_rank / out["single_problem_fp64"]["value"]
        out["speedup_over_mixed_single_problem"] = value_rank / out["single_problem_mixed"]["value"]
    return out


def cpu_baseline(args, bounded_seconds=12.0, steps=None):
    """The oracle as it stands (single thread, FP64) on a bounded sample of the
    same workload: accepted time steps from the initial state."""
    import oracle as O
    from paper_2104_11404_gb300 import workloads as W
    cfg = W.CONFIGS[WORKLOAD]
    o = O.Oracle(dim=cfg["dim"], nx=cfg["n"][0], ny=cfg["n"][1], nz=cfg["n"][2],
                 lo=list(cfg["lo"]), hi=list(cfg["hi"]), order=cfg["order"], problem=cfg["problem"],
                 gamma=cfg["gamma"], visc=cfg["visc"], source=cfg.get("source", 1),
                 cfl=cfg.get("cfl", 0.5))
    v, e, x = o.init_state()
    N = o.nv * 2 + o.ne
    total, t0 = 0, time.time()
    dt = 0.0
    while time.time() - t0 < bounded_seconds and (steps is None or total < steps):
        stats, log, st = o.run(cfg["t_final"], v, e, x, dt=dt, max_steps=5)
        dt = stats["dt"]
        total += stats["steps"]
    el = time.time() - t0
    return {"value": N * total / el, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle",
            "sample": "%d accepted RK2-average steps of the 64x64 Taylor-Green workload from t = 0, "
                      "single-thread FP64 C oracle, %.1f s" % (total, el)}


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores, each bench step a
    bounded sample (CHUNK_REF accepted time steps) of the same workload."""
    world, rank, local = _dist()
    if rank != 0:
        return None
    import oracle as O
    from paper_2104_11404_gb300 import workloads as W
    O.lib()
    cfg = W.CONFIGS[WORKLOAD]
    o = O.Oracle(dim=cfg["dim"], nx=cfg["n"][0], ny=cfg["n"][1], nz=cfg["n"][2],
                 lo=list(cfg["lo"]), hi=list(cfg["hi"]), order=cfg["order"], problem=cfg["problem"],
                 gamma=cfg["gamma"], visc=cfg["visc"], source=cfg.get("source", 1),
                 cfl=cfg.get("cfl", 0.5))
    v, e, x = o.init_state()
    N = 2 * o.nv + o.ne
    chunk = 5
    dt = 0.0
    for _ in range(args.warmup):
        stats, _, _ = o.run(cfg["t_final"], v, e, x, dt=dt, max_steps=chunk)
        dt = stats["dt"]
    t0 = time.time()
    total = 0
    for _ in range(args.steps):
        stats, _, _ = o.run(cfg["t_final"], v, e, x, dt=dt, max_steps=chunk)
        dt = stats["dt"]
        total += stats["steps"]
    el = time.time() - t0
    value = N * total / el
    return {"metric": "Lagrangian step DOF-updates/s; mixed/batched vs FP64 GPU at stated rel. error",
            "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "2D Taylor-Green vortex 64x64 Q2/Q1, AV on, CFL 0.1",
                       "dofs_per_instance": N, "time_steps_per_bench_step": chunk},
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle",
                             "sample": "%d bench steps of %d accepted time steps" % (args.steps, chunk)},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched sweep")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (2D blast 8x8, 3D blast 32^3, Gresho 256^2 Q3)")
    ap.add_argument("--direct-launch", action="store_true",
                    help="launch the step's kernels one by one instead of one CUDA graph per "
                         "attempt (kernel profilers cannot see kernels inside graphs with "
                         "conditional nodes)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    line = run_reference(args) if args.impl == "reference" else run_native(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
