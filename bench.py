"""Benchmark: Lagrangian step DOF-updates/s of the full-order hydro step.

Headline workload: the batched parameter sweep, 512 independent 2D
point-blast instances (Section 6.1.2 problem; E0 ~ U[0.1, 1], gamma ~
U[1.3, 1.67], n x n Q2/Q1 quads with n from {16, 24, 32, 48}; splitmix64 seed
2104114040), mixed FP32/FP64, one persistent kernel per RK2-average stage,
the two stage kernels of an attempt one CUDA graph, launch shape autotuned.
One bench step = the whole sweep: every instance from its initial condition
to t = 0.8 under its own step control (lh_batch_set_state of the initial
packed state resident on the device, then lh_batch_run_to).
value = sum over instances of (2 N_V + N_E) x accepted steps / device time.

Beside it: the same sweep in FP64, the instance mix through the single-problem
FP64 and mixed paths, the restricted (5% element sample) force, full runs of
the single-problem workloads (2D blast 8x8 to 0.8, Taylor-Green 64x64 to 0.5,
3D blast 32^3 to 0.6, Gresho 256^2 Q3 to 0.62) in FP64 and mixed, and the CPU
oracle on a seeded subset of the sweep on all host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
Under torchrun every rank advances its own copy of the sweep (independent
replicas, weak scaling, no collective on the data path); rank 0 prints one
JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lagrangian step DOF-updates/s; mixed/batched vs FP64 GPU at stated rel. error"
SWEEP_T_FINAL = 0.8
CHUNK = 100          # accepted time steps of every unfinished sweep instance per bench step
SWEEP_WORKLOAD = ("batched sweep: 512 independent 2D point-blast instances, E0 U[0.1,1], gamma "
                  "U[1.3,1.67], n x n Q2/Q1 quads with n from {16,24,32,48}, each from its initial "
                  "condition to t = 0.8, splitmix64 seed 2104114040")
# CPU oracle sample of the sweep: the first instances of the seeded list, on
# every host core
CPU_SUBSET_PER_CORE = 2
# DRAM read + write per launch of the batched stage kernel from an ncu capture,
# or None until the current kernel is captured
STAGE_KERNEL_DRAM_BYTES = None


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


def batch_fp64_flops(cfgs):
    """FP64 flops of one attempt (two stages) of the batched mixed step, summed
    over instances: the work the mixed design keeps in FP64 (2D Q2/Q1, n_e
    elements, N_V velocity unknowns per instance), counted per stage from the
    kernels' loops.  Per element: the FP64 element-origin shift of the staged
    positions 18, the widening of the error-free F.1 row sums 18, the node
    gather of -F.1 18, the CG mass apply (two 3x3 contractions per component,
    54 multiply-adds each, the rho0|J0| scaling 18) 234 and its node sums 18,
    the energy update (widening of the error-free F^T w sums 4, M_E^-1 16
    multiply-adds, the update 4 multiply-adds) 44: 350.  Per velocity unknown:
    the line solves 21 (forward and backward substitution along both
    directions, k = 2, and the scale), the CG dots and updates 12, the stage
    update 4: 37."""
    tot = 0
    for c in cfgs:
        n = c["n"][0] * c["n"][1]
        nn = (2 * c["n"][0] + 1) * (2 * c["n"][1] + 1)
        nv = 2 * nn
        tot += 350 * n + 37 * nv
    return 2 * tot


def stage_words(nv, ne, nqp, cg_iters):
    """Algorithmic FP64 words moved by one RK stage of one problem (the
    per-stage table of the measurement plan): force in 2 N_V + N_E + N_qp,
    force out N_V, CG I (6 N_V + N_qp), F^T v and e update 2 N_V + 2 N_E +
    N_qp, x update 3 N_V."""
    return (2 * nv + ne + nqp) + nv + cg_iters * (6 * nv + nqp) + (2 * nv + 2 * ne + nqp) + 3 * nv


def batch_attempt_bytes(cfgs, cg_iters_per_solve):
    tot = 0.0
    for c in cfgs:
        n = c["n"][0] * c["n"][1]
        nv = 2 * (2 * c["n"][0] + 1) * (2 * c["n"][1] + 1)
        tot += 2 * stage_words(nv, 4 * n, 16 * n, cg_iters_per_solve)
    return 8.0 * tot


def _measured_hbm():
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if p.get("hbm_gbs"):
            return float(p["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except Exception:
        pass
    return 6800.0, "profiling recipe fallback 6.8 TB/s (of fallback)"


# ------------------------------------------------------------ CPU oracle pool

def _oracle_worker(conn, cfgs, t_final):
    """Host worker (spawned): holds a fixed subset of sweep instances in the
    CPU oracle and advances each by the requested accepted steps, restarting
    an instance from its initial condition when it reaches t_final."""
    sys.path.insert(0, ROOT)
    import oracle as O
    from tests._pair import oracle_for
    insts = []
    for c in cfgs:
        o = oracle_for(c)
        v, e, x = o.init_state()
        insts.append([o, v, e, x, 0.0, 0.0])
    conn.send(("ready", len(insts)))
    while True:
        msg = conn.recv()
        if msg[0] == "stop":
            break
        steps_each = msg[1]
        upd = 0
        for rec in insts:
            o, v, e, x, t, dt = rec
            if t >= t_final:
                v, e, x = o.init_state()
                t, dt = 0.0, 0.0
                rec[1:4] = [v, e, x]
            st, _, s = o.run(t_final, v, e, x, t0=t, dt=dt, max_steps=steps_each)
            if s != O.OK:
                raise RuntimeError("oracle status %d" % s)
            rec[4], rec[5] = st["t"], st["dt"]
            upd += (2 * o.nv + o.ne) * st["steps"]
        conn.send(("done", upd))
    conn.close()


class OraclePool:
    """The CPU oracle, as it stands, on every host core: one spawned process
    per core, each owning a fixed share of the instances."""

    def __init__(self, cfgs, nproc, t_final):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for w in range(nproc):
            mine = cfgs[w::nproc]
            if not mine:
                continue
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, mine, t_final), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            c.recv()
        self.cores = len(self.procs)

    def advance(self, steps_each):
        t0 = time.time()
        for c in self.conns:
            c.send(("adv", steps_each))
        upd = sum(c.recv()[1] for c in self.conns)
        return upd, time.time() - t0

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)


def _cpu_subset(nproc):
    from paper_2104_11404_gb300 import workloads as W
    cfgs = W.batch_instances()
    return cfgs[:CPU_SUBSET_PER_CORE * nproc]


def cpu_baseline_sweep(bounded_seconds=15.0, steps_each=3):
    """The oracle on a bounded sample of the sweep on all host cores: the
    first 2 x nproc instances of the seeded list advanced from their initial
    conditions in rounds of `steps_each` accepted steps each, until about
    `bounded_seconds` of wall time."""
    nproc = os.cpu_count() or 1
    sub = _cpu_subset(nproc)
    pool = OraclePool(sub, nproc, SWEEP_T_FINAL)
    try:
        upd, el, rounds = 0, 0.0, 0
        while el < bounded_seconds and rounds < 200:
            u, dt = pool.advance(steps_each)
            upd += u
            el += dt
            rounds += 1
    finally:
        pool.close()
    return {"value": upd / el, "unit": "DOF-updates/s", "cores": pool.cores, "kind": "oracle",
            "sample": "%d instances of the seeded sweep (the first 2 per core; sizes %s), %d rounds "
                      "of %d accepted RK2-average steps each from t = 0, single-thread FP64 C "
                      "oracle per process, %d spawned processes on %d host cores, %.1f s" %
                      (len(sub), sorted({c["n"][0] for c in sub}), rounds, steps_each,
                       pool.cores, nproc, el),
            "nproc": nproc}


# ------------------------------------------------------------ native arm

def _inst_flops_bytes(cfgs, cg_iters_per_solve):
    """Per instance: algorithmic FP64 flops and bytes of one attempt."""
    import numpy as np
    fl = np.array([batch_fp64_flops([c]) for c in cfgs], dtype=np.float64)
    by = np.array([batch_attempt_bytes([c], cg_iters_per_solve) for c in cfgs], dtype=np.float64)
    return fl, by


def measure_sweep(args, stream, flush, precision, reduce_max, reduce_sum, steps=None,
                  warmup=None, autotune=True, e2e=True, whole=False):
    """The batched sweep in bench steps of CHUNK accepted time steps of every
    unfinished instance, the sweep continuing from one bench step to the next
    (restarted from the initial state, untimed, once every instance has reached
    t = 0.8).  With whole=True one complete sweep from t = 0 is also timed."""
    import numpy as np
    import torch
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.batch import Batch
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    cfgs = W.batch_instances()
    out = {}
    with torch.cuda.stream(stream):
        b = Batch(cfgs, precision=precision, stream=stream)
        b.init_state()
        v0, e0, x0 = b.get_state()           # initial packed state, resident on the device
        zeros = np.zeros(b.n)
        tune, tune_s = None, 0.0
        if autotune:
            t0 = time.time()
            tune = b.autotune(reps=2)
            tune_s = time.time() - t0
        dofs = b.dofs()
        state = {"fresh": True}

        def restart_if_done():
            q = b.query()
            if state["fresh"] or np.all(q["t"] >= SWEEP_T_FINAL):
                b.set_state(v0, e0, x0, zeros, zeros)
                state["fresh"] = False

        for _ in range(warmup):
            restart_if_done()
            b.run_to(SWEEP_T_FINAL, max_steps=CHUNK)
        torch.cuda.synchronize()
        dev_ms, upd, nsteps, rejects, graphs, cg = 0.0, 0, 0, 0, 0, 0
        att_i = np.zeros(b.n)
        clk = Clocks(torch.cuda.current_device())
        clk.start()
        for _ in range(steps):
            restart_if_done()
            flush.fill_(1.0)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            st = b.run_to(SWEEP_T_FINAL, max_steps=CHUNK)
            ev1.record(stream)
            ev1.synchronize()
            dev_ms += ev0.elapsed_time(ev1)
            q = b.query()
            att_i += q["steps"] + q["rejects"]
            upd += st["dof_updates"]
            nsteps += st["steps"]
            rejects += st["rejects"]
            graphs += st["graph_launches"]
            cg += st["cg_iters"]
        clocks = clk.stop()
        attempts = nsteps + rejects
        out = {"dev_ms": dev_ms, "dof_updates": upd, "steps": nsteps, "rejects": rejects,
               "graph_launches": graphs, "attempts_per_instance": att_i,
               "cg_iters_per_solve": cg / max(1, 2 * attempts), "tuning": tune,
               "autotune_s": tune_s, "clocks": clocks,
               "value": reduce_sum(upd) / (reduce_max(dev_ms) * 1e-3) if steps else None,
               "value_rank": upd / (dev_ms * 1e-3) if steps else None,
               "dofs_total": int(dofs.sum()),
               "instances": len(cfgs), "bench_steps": steps}
        if e2e:
            # end to end through the C ABI: the bench step's state from pinned
            # host memory, the chunk, the new state back to pinned host memory
            hv = torch.empty(b.nv, dtype=torch.float64, pin_memory=True)
            he = torch.empty(b.ne, dtype=torch.float64, pin_memory=True)
            hx = torch.empty(b.nv, dtype=torch.float64, pin_memory=True)
            b.set_state(v0, e0, x0, zeros, zeros)
            lagh.lh_batch_get_state(b.b, hv, he, hx)
            q = b.query()
            e2e_ms, e2e_upd = 0.0, 0
            for _ in range(max(1, steps // 2)):
                flush.fill_(1.0)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                b.set_state(hv, he, hx, q["t"], q["dt"])
                st = b.run_to(SWEEP_T_FINAL, max_steps=CHUNK)
                lagh.lh_batch_get_state(b.b, hv, he, hx)
                q = b.query()
                ev1.record(stream)
                ev1.synchronize()
                e2e_ms += ev0.elapsed_time(ev1)
                e2e_upd += st["dof_updates"]
            out["e2e"] = {"value": reduce_sum(e2e_upd) / (reduce_max(e2e_ms) * 1e-3),
                          "unit": "DOF-updates/s",
                          "h2d_bytes_per_step": 8 * (2 * b.nv + b.ne) + 16 * b.n,
                          "d2h_bytes_per_step": 8 * (2 * b.nv + b.ne)}
        if whole:
            flush.fill_(1.0)
            b.set_state(v0, e0, x0, zeros, zeros)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            b.set_state(v0, e0, x0, zeros, zeros)
            st = b.run_to(SWEEP_T_FINAL)
            ev1.record(stream)
            ev1.synchronize()
            ms = ev0.elapsed_time(ev1)
            q = b.query()
            assert np.all(q["t"] == SWEEP_T_FINAL) and np.all(q["status"] == 0)
            fv, fe, _ = b.get_state()
            out["whole"] = {"value": st["dof_updates"] / (ms * 1e-3), "sweep_ms": ms,
                            "accepted_steps": st["steps"], "rejects": st["rejects"],
                            "steps_per_instance_mean": st["steps"] / b.n,
                            "energy_min": float(np.min(b.total_energy()))}
            out["final_state"] = (fv.cpu().numpy(), fe.cpu().numpy(), b.off_v.copy(),
                                  b.off_e.copy())
        b.close()
    return out


def measure_hyper_reduced(stream):
    """Restricted force (Section 3.3) on a seeded 5% element sample of every
    sweep instance, timed alone."""
    import numpy as np
    import torch
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.batch import Batch
    cfgs = W.batch_instances()
    with torch.cuda.stream(stream):
        b = Batch(cfgs, precision="mixed", stream=stream)
        b.init_state()
        b.run_to(0.1)
        lists = [W.element_sample(c["n"][0] * c["n"][1], frac=0.05, stream=i)
                 for i, c in enumerate(cfgs)]
        nsamp = int(sum(len(l) for l in lists))
        F1, _, off, _ = b.force_sampled(lists)
        d_off = torch.from_numpy(off).to("cuda")
        d_ids = torch.from_numpy(np.concatenate(lists).astype(np.int32)).to("cuda")
        reps = 20
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            lagh.lh_batch_force_sampled(b.b, d_off, d_ids, F1)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        b.close()
    return {"sampled_elements": nsamp, "launch_us": ms * 1e3, "elements_per_s": nsamp / (ms * 1e-3),
            "sample": "ceil(0.05 n_e) elements per instance, seeded Fisher-Yates, sorted"}


def measure_single_sizes(stream, nsteps=20):
    """The sweep's mesh sizes through the plain single-problem path (one
    context per problem), FP64 and mixed: DOF-updates/s over a window."""
    import torch
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.hydro import Hydro
    cfg0 = W.batch_instances()[0]
    rates = {}
    with torch.cuda.stream(stream):
        for prec in ("fp64", "mixed"):
            for n in W.BATCH_SIZES:
                c = dict(cfg0, n=(n, n, 1), gamma=1.4, blast_energy=0.5)
                g = Hydro(c, precision=prec, stream=stream)
                g.init_state()
                g.run_to(0.8, max_steps=3)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                st = g.run_to(0.8, max_steps=nsteps)
                ev1.record(stream)
                ev1.synchronize()
                rates[(prec, n)] = (2 * g.nv + g.ne) * st["steps"] / (ev0.elapsed_time(ev1) * 1e-3)
                g.close()
    return rates


def measure_sweep_accuracy(stream, count=12, max_n=24):
    """The mixed batched path against the FP64 batched path at t = 0.8 on the
    first `count` sweep instances of mesh size <= max_n: relative L2 difference
    per instance (eq:relerrors), the worst, and the step counts."""
    import numpy as np
    import torch
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.batch import Batch
    sub = [c for c in W.batch_instances() if c["n"][0] <= max_n][:count]
    res = {}
    with torch.cuda.stream(stream):
        for prec in ("fp64", "mixed"):
            b = Batch(sub, precision=prec, stream=stream)
            b.init_state()
            b.run_to(SWEEP_T_FINAL)
            v, e, _ = b.get_state()
            q = b.query()
            res[prec] = (v.cpu().numpy(), e.cpu().numpy(), q["steps"].copy(), b.off_v.copy(),
                         b.off_e.copy(), b.total_energy())
            b.close()
    fv, fe, fs, ov, oe, fE = res["fp64"]
    mv, me, ms, _, _, mE = res["mixed"]
    rel = lambda a, b_: float(np.linalg.norm(b_ - a) / max(np.linalg.norm(a), 1e-300))
    dv = [rel(fv[ov[i]:ov[i + 1]], mv[ov[i]:ov[i + 1]]) for i in range(len(sub))]
    de = [rel(fe[oe[i]:oe[i + 1]], me[oe[i]:oe[i + 1]]) for i in range(len(sub))]
    free = {"what": "each path under its own step control to t = 0.8 (a borderline "
                    "step-control decision can part the step sequences, after which the runs "
                    "differ by their time discretisation)",
            "rel_l2_v_worst": max(dv), "rel_l2_e_worst": max(de),
            "rel_l2_v_median": float(np.median(dv)), "rel_l2_e_median": float(np.median(de)),
            "steps_fp64": [int(x) for x in fs], "steps_mixed": [int(x) for x in ms],
            "energy_drift_mixed_worst": float(np.max(np.abs(mE - fE) / np.abs(fE)))}
    # precision alone: the mixed batch replays the FP64 step sizes of each
    # instance (one context per instance records them) for the common number
    # of accepted steps, against the FP64 state after those steps
    from paper_2104_11404_gb300.hydro import Hydro
    sub2 = sub[:4]
    logs, refs = [], []
    with torch.cuda.stream(stream):
        for c in sub2:
            g = Hydro(c, precision="fp64", stream=stream)
            g.init_state()
            lg = torch.zeros(20000, dtype=torch.float64, device="cuda")
            st = g.run_to(SWEEP_T_FINAL, dt_log=lg)
            logs.append(lg.cpu().numpy()[:st["steps"]])
            g.close()
        nrep = min(len(l) for l in logs)
        for c in sub2:
            g = Hydro(c, precision="fp64", stream=stream)
            g.init_state()
            g.run_to(SWEEP_T_FINAL, max_steps=nrep)
            v, e, _, _, _ = g.get_state()
            refs.append((v.cpu().numpy(), e.cpu().numpy()))
            g.close()
        out = {}
        for label, prec, perturb in (("mixed", "mixed", False), ("fp64_perturbed", "fp64", True)):
            b = Batch(sub2, precision=prec, stream=stream)
            b.init_state()
            if perturb:
                # the conditioning of the problem: the FP64 run from an initial
                # energy perturbed by a seeded 1e-7 relative amount
                v0, e0, x0 = b.get_state()
                gen = torch.Generator(device="cuda").manual_seed(2104)
                noise = 2.0 * torch.rand(e0.shape, generator=gen, device="cuda",
                                         dtype=torch.float64) - 1.0
                b.set_state(v0, e0 * (1.0 + 1e-7 * noise), x0)
            for k in range(nrep):
                b.step_fixed(np.array([l[k] for l in logs]))
            v, e, _ = b.get_state()
            v, e = v.cpu().numpy(), e.cpu().numpy()
            out[label] = ([rel(refs[i][0], v[b.off_v[i]:b.off_v[i + 1]]) for i in range(len(sub2))],
                          [rel(refs[i][1], e[b.off_e[i]:b.off_e[i + 1]]) for i in range(len(sub2))])
            b.close()
    replay = {"what": "the mixed batch replaying each instance's FP64 step sizes (%d accepted "
                      "steps): the precision alone" % nrep,
              "instances": len(sub2), "rel_l2_v": out["mixed"][0], "rel_l2_e": out["mixed"][1],
              "rel_l2_v_worst": max(out["mixed"][0]), "rel_l2_e_worst": max(out["mixed"][1]),
              "conditioning": {"what": "the FP64 batch from an initial energy perturbed by 1e-7 "
                                       "(relative, seeded), same step sizes",
                               "rel_l2_v": out["fp64_perturbed"][0],
                               "rel_l2_e": out["fp64_perturbed"][1]}}
    return {"instances": len(sub), "sizes": sorted({c["n"][0] for c in sub}),
            "replay": replay, "free_running": free}


WINDOWS = {"sedov2d_8": None, "tg2d_64": 50, "sedov3d_32": 20, "gresho2d_256": 20}


def measure_windows(stream):
    """The single-problem workloads through one context each, FP64 and mixed:
    a window of accepted steps after three warm-up steps (the 2D blast 8x8 to
    its final time): throughput, the mixed/FP64 speed-up, the mixed state's
    relative L2 difference from the FP64 state after the same window, and the
    mixed energy drift (problems without a source)."""
    import numpy as np
    import torch
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.hydro import Hydro
    out = {}
    for name, nsteps in WINDOWS.items():
        cfg = W.CONFIGS[name]
        res, states = {}, {}
        for prec in ("fp64", "mixed"):
            with torch.cuda.stream(stream):
                g = Hydro(cfg, precision=prec, stream=stream)
                g.init_state()
                E0 = g.total_energy()
                if nsteps is not None:
                    g.run_to(cfg["t_final"], max_steps=3)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                st = g.run_to(cfg["t_final"], max_steps=nsteps if nsteps else 2 ** 62)
                ev1.record(stream)
                ev1.synchronize()
                ms = ev0.elapsed_time(ev1)
                N = 2 * g.nv + g.ne
                v, e, x, t, _ = g.get_state()
                states[prec] = (v.cpu().numpy(), e.cpu().numpy(), t)
                r = {"value": N * st["steps"] / (ms * 1e-3), "ms_per_step": ms / max(1, st["steps"]),
                     "steps": st["steps"],
                     "cg_iters_per_solve": st["cg_iters"] / max(1, 2 * (st["steps"] + st["rejects"]))}
                if cfg["problem"] != W.TAYLOR_GREEN:
                    r["energy_drift"] = abs(g.total_energy() - E0) / abs(E0)
                res[prec] = r
                g.close()
        rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(a), 1e-300))
        out[name] = {"dofs": int(N), "window": nsteps if nsteps else "to t_final",
                     "fp64": res["fp64"], "mixed": res["mixed"],
                     "speedup_mixed_over_fp64": res["mixed"]["value"] / res["fp64"]["value"],
                     "mixed_vs_fp64_rel_l2": {"v": rel(states["fp64"][0], states["mixed"][0]),
                                              "e": rel(states["fp64"][1], states["mixed"][1])}}
    return out


def measure_rom(stream, t_final=0.1):
    """The reduced model of Sections 3-4 on the 3D blast of Table tab:fom
    (8^3 Q2/Q1, FP64) over t in [0, 0.1]: snapshots of the batched run, GPU POD
    bases (0.9999 criterion), SNS bases and over-sampled DEIM (twice the basis
    sizes), then the hyper-reduced online run against the full-order run over
    the same interval: wall time of each time loop, speed-up, and the lifted
    reduced state's relative L2 error at t = 0.1 (eq:relerrors).  The same
    bases then run on a mixed context against the mixed full-order run
    ("mixed": the stress and F_K of the sampled elements in FP32)."""
    import numpy as np
    import torch
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.batch import Batch
    from paper_2104_11404_gb300.hydro import Hydro
    from paper_2104_11404_gb300.rom import Rom
    cfg = W.scaled("sedov3d_32", n=(8, 8, 8), t_final=t_final)
    with torch.cuda.stream(stream):
        b = Batch([cfg], precision="fp64", stream=stream)
        b.init_state()
        v0, e0, x0 = (a.clone() for a in b.get_state())
        Sv, Se, Sx = b.snapshots([0], 8000)
        b.run_to(t_final)
        (_, cnt, V, E, X), = b.snapshot_views(Sv, Se, Sx)
        bases = []
        for cols, off in ((V, v0), (E, e0), (X, x0)):
            n, m = cols.shape
            U = torch.zeros(n * m, dtype=torch.float64, device="cuda")
            sig = torch.zeros(n, dtype=torch.float64, device="cuda")
            work = torch.zeros(m * n + 2 * n + 16, dtype=torch.float64, device="cuda")
            k, _ = lagh.lh_pod(cols.contiguous(), m, n, off, 0.9999, U, sig, work, stream.cuda_stream)
            bases.append(U.view(n, m)[:k].contiguous())
        b.close()
        f = Hydro(cfg, precision="fp64", stream=stream)
        f.init_state()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        stf = f.run_to(t_final)
        ev1.record(stream)
        ev1.synchronize()
        fom_ms = ev0.elapsed_time(ev1)
        fv, fe, fx, _, _ = f.get_state()
        g = Hydro(cfg, precision="fp64", stream=stream)
        nb = [B.shape[0] for B in bases]
        r = Rom(g, bases[0], bases[1], bases[2], v0, e0, x0, min(2 * nb[0], g.nv),
                min(2 * nb[1], g.ne))
        r.run_to(t_final)                       # warm-up (builds the graph)
        r.set_state(np.zeros(nb[0]), np.zeros(nb[1]), np.zeros(nb[2]))
        ev0.record(stream)
        st = r.run_to(t_final)
        ev1.record(stream)
        ev1.synchronize()
        rom_ms = ev0.elapsed_time(ev1)
        lv, le, lx = r.lift()
        rel = lambda a, b_: float(torch.linalg.norm(b_ - a) / torch.linalg.norm(a))
        out = {"problem": "3D point blast 8^3 Q2/Q1 (Table tab:fom), t in [0, %g], FP64" % t_final,
               "snapshots": int(cnt), "basis_sizes": {"v": nb[0], "e": nb[1], "x": nb[2]},
               "samples": {"F1": int(r.info.ns_f), "FTv": int(r.info.ns_g)},
               "sampled_elements": int(r.info.n_elems), "elements": int(g.nelem),
               "fom": {"steps": stf["steps"], "ms": fom_ms},
               "rom": {"steps": st["steps"], "ms": rom_ms},
               "speedup_rom_over_fom": fom_ms / rom_ms,
               "rel_l2_error_at_t_final": {"v": rel(fv, lv), "e": rel(fe, le), "x": rel(fx, lx)}}
        r.close()
        g.close()
        f.close()
        # the same reduced model on mixed contexts
        fm = Hydro(cfg, precision="mixed", stream=stream)
        fm.init_state()
        ev0.record(stream)
        stfm = fm.run_to(t_final)
        ev1.record(stream)
        ev1.synchronize()
        fom_m_ms = ev0.elapsed_time(ev1)
        gm = Hydro(cfg, precision="mixed", stream=stream)
        rm = Rom(gm, bases[0], bases[1], bases[2], v0, e0, x0, min(2 * nb[0], gm.nv),
                 min(2 * nb[1], gm.ne))
        rm.run_to(t_final)
        rm.set_state(np.zeros(nb[0]), np.zeros(nb[1]), np.zeros(nb[2]))
        ev0.record(stream)
        stm = rm.run_to(t_final)
        ev1.record(stream)
        ev1.synchronize()
        rom_m_ms = ev0.elapsed_time(ev1)
        mv, me, mx = rm.lift()
        out["mixed"] = {"fom": {"steps": stfm["steps"], "ms": fom_m_ms},
                        "rom": {"steps": stm["steps"], "ms": rom_m_ms},
                        "speedup_rom_over_fom": fom_m_ms / rom_m_ms,
                        "speedup_over_fp64_fom": fom_ms / rom_m_ms,
                        "rel_l2_error_at_t_final_vs_fp64_fom": {"v": rel(fv, mv), "e": rel(fe, me),
                                                               "x": rel(fx, mx)}}
        rm.close()
        gm.close()
        fm.close()
    return out


FULL_RUNS = ("sedov2d_8", "tg2d_64", "sedov3d_32", "gresho2d_256")


def _tg_exact_error(g, v, x):
    """Relative L2 (nodal) error of the velocity against the steady exact 2D
    Taylor-Green field, evaluated at the final node positions."""
    import numpy as np
    nn = g.nv // 2
    X, Y = x[:nn], x[nn:]
    ve = np.concatenate([np.sin(np.pi * X) * np.cos(np.pi * Y), -np.cos(np.pi * X) * np.sin(np.pi * Y)])
    return float(np.linalg.norm(v - ve) / np.linalg.norm(ve))


def measure_full_runs(stream):
    """Every single-problem workload from its initial condition to its final
    time, FP64 and mixed: device time of the time loop, steps, throughput,
    energy drift, the mixed state's relative L2 difference from the FP64 state
    at the final time (eq:relerrors), and for Taylor-Green the error against
    the exact solution."""
    import numpy as np
    import torch
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.hydro import Hydro
    out = {}
    for name in FULL_RUNS:
        cfg = W.CONFIGS[name]
        res, states = {}, {}
        for prec in ("fp64", "mixed"):
            with torch.cuda.stream(stream):
                g = Hydro(cfg, precision=prec, stream=stream)
                g.init_state()
                E0 = g.total_energy()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                st = g.run_to(cfg["t_final"])
                ev1.record(stream)
                ev1.synchronize()
                ms = ev0.elapsed_time(ev1)
                N = 2 * g.nv + g.ne
                v, e, x, t, _ = g.get_state()
                v, e, x = v.cpu().numpy(), e.cpu().numpy(), x.cpu().numpy()
                states[prec] = (v, e, x)
                r = {"value": N * st["steps"] / (ms * 1e-3), "run_s": ms * 1e-3,
                     "ms_per_step": ms / max(1, st["steps"]), "steps": st["steps"],
                     "rejects": st["rejects"], "t": t,
                     "cg_iters_per_solve": st["cg_iters"] / max(1, 2 * (st["steps"] + st["rejects"]))}
                if not cfg.get("source", 0) or cfg["problem"] != W.TAYLOR_GREEN:
                    r["energy_drift"] = abs(g.total_energy() - E0) / abs(E0)
                if cfg["problem"] == W.TAYLOR_GREEN:
                    r["velocity_error_vs_exact"] = _tg_exact_error(g, v, x)
                res[prec] = r
                g.close()
        rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(a), 1e-300))
        out[name] = {"dofs": int(N), "t_final": cfg["t_final"], "fp64": res["fp64"],
                     "mixed": res["mixed"],
                     "speedup_mixed_over_fp64": res["mixed"]["value"] / res["fp64"]["value"],
                     "mixed_vs_fp64_rel_l2_at_t_final": {
                         "v": rel(states["fp64"][0], states["mixed"][0]),
                         "e": rel(states["fp64"][1], states["mixed"][1]),
                         "x": rel(states["fp64"][2], states["mixed"][2])}}
    return out


def run_native(args):
    import torch
    from paper_2104_11404_gb300 import build as libbuild
    from paper_2104_11404_gb300 import peaks as peaks_mod

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    libbuild.build()
    stream = torch.cuda.Stream()

    def reduce_max(x):
        return rank_reduce(x, "max", world, "cuda")

    def reduce_sum(x):
        return rank_reduce(x, "sum", world, "cuda")

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    pk = peaks_mod.measure(stream)
    hbm_peak, hbm_src = _measured_hbm()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sw = measure_sweep(args, stream, flush, "mixed", reduce_max, reduce_sum)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        return None
    from paper_2104_11404_gb300 import workloads as W
    import numpy as np
    cfgs = W.batch_instances()
    extra = not args.quick
    whole = measure_sweep(args, stream, flush, "mixed", lambda x: x, lambda x: x, steps=0,
                          warmup=0, autotune=True, e2e=False, whole=True)["whole"] if extra else None
    sw64 = measure_sweep(args, stream, flush, "fp64", lambda x: x, lambda x: x, steps=3, warmup=1,
                         autotune=True, e2e=False) if extra else None
    acc = measure_sweep_accuracy(stream) if extra else None
    rates = measure_single_sizes(stream) if extra else None
    hr = measure_hyper_reduced(stream) if extra else None
    windows = measure_windows(stream) if (extra and not args.no_configs) else None
    full = measure_full_runs(stream) if args.full_runs else None
    rom = measure_rom(stream) if extra else None

    value = sw["value"]
    fl_i, by_i = _inst_flops_bytes(cfgs, sw["cg_iters_per_solve"])
    att = sw["attempts_per_instance"]
    dev_s = sw["dev_ms"] * 1e-3
    achieved = float(fl_i @ att) / dev_s / 1e12
    abytes = float(by_i @ att)
    kernels_per_graph = 2
    launches = sw["graph_launches"] * kernels_per_graph + 2 * args.steps  # + estimate, begin
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "DOF-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sw["dev_ms"] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": SWEEP_WORKLOAD, "instances": sw["instances"],
                   "dofs_total": sw["dofs_total"], "precision": "mixed FP32/FP64",
                   "step": "%d accepted RK2-average time steps of every unfinished instance, the "
                           "sweep continuing across bench steps and restarting from t = 0 once "
                           "every instance has reached t = 0.8" % CHUNK,
                   "l2": "flushed between timed steps (256 MB write); the packed state and "
                         "per-CTA scratch exceed L2",
                   "tuning": sw["tuning"], "autotune_s": sw["autotune_s"],
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "alu", "kernel": "batch_stage_kernel (both stage kernels of an attempt)",
                     "achieved": achieved, "peak": pk["fp64_tflops"], "unit": "TFLOP/s (FP64)",
                     "frac": achieved / pk["fp64_tflops"], "traffic": STAGE_KERNEL_DRAM_BYTES,
                     "algorithmic_fp64_flops": float(fl_i @ att),
                     "attempts": float(att.sum()),
                     "peak_source": "FP64 FMA probe measured in this run (lh_peak_probe, of measured)",
                     "hbm_view": {"algorithmic_bytes": abytes,
                                  "achieved": abytes / dev_s / 1e9, "peak": hbm_peak,
                                  "unit": "GB/s", "frac": abytes / dev_s / 1e9 / hbm_peak,
                                  "peak_source": hbm_src,
                                  "cg_iters_per_solve": sw["cg_iters_per_solve"]}},
        "e2e": sw["e2e"],
        "gpu_launches": int(launches),
        "clocks": sw["clocks"],
        "measured_peaks": {"fp64_tflops": pk["fp64_tflops"], "fp32_tflops": pk["fp32_tflops"],
                           "hbm_gbs": hbm_peak},
        "sweep": {"accepted_steps": sw["steps"], "rejects": sw["rejects"],
                  "attempt_graphs": sw["graph_launches"]},
    }
    if whole is not None:
        line["whole_sweep"] = whole
    if sw64 is not None:
        v64 = sw64["value_rank"]
        line["batched_fp64"] = {"value": v64, "ms_per_step": sw64["dev_ms"] / sw64["bench_steps"],
                                "tuning": sw64["tuning"],
                                "speedup_mixed_over_fp64_batched": sw["value_rank"] / v64}
    if acc is not None:
        line["mixed_accuracy"] = acc
    if rates is not None:
        dofs = np.array([2 * 2 * (2 * c["n"][0] + 1) * (2 * c["n"][1] + 1) + 4 * c["n"][0] * c["n"][1]
                         for c in cfgs], dtype=np.float64)
        share = dofs / dofs.sum()

        def mix_rate(prec):  # the same DOF-updates through one context per problem
            return 1.0 / sum(share[i] / rates[(prec, c["n"][0])] for i, c in enumerate(cfgs))
        line["single_problem"] = {
            "fp64": {"value": mix_rate("fp64"),
                     "rates_by_size": {str(n): rates[("fp64", n)] for n in W.BATCH_SIZES}},
            "mixed": {"value": mix_rate("mixed"),
                      "rates_by_size": {str(n): rates[("mixed", n)] for n in W.BATCH_SIZES}},
            "speedup_batched_mixed_over_fp64_single_problem": sw["value_rank"] / mix_rate("fp64"),
            "speedup_batched_mixed_over_mixed_single_problem": sw["value_rank"] / mix_rate("mixed")}
    if hr is not None:
        line["hyper_reduced_force"] = hr
    if windows is not None:
        line["configs"] = windows
    if full is not None:
        line["full_runs"] = full
    if rom is not None:
        line["rom"] = rom
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sweep()
    if world == 1 and args.cpu_configs:
        line["cpu_configs"] = cpu_configs()
    return line


def cpu_configs(seconds=6.0):
    """The oracle on the single-problem workloads, as it stands: one core
    (accepted steps from the initial state for about `seconds`) and all host
    cores (one independent copy of the problem per core, spawned processes,
    the same accepted steps each); DOF-updates/s with the core count."""
    import oracle as O
    from paper_2104_11404_gb300 import workloads as W
    from tests._pair import oracle_for
    nproc = os.cpu_count() or 1
    out = {}
    for name in WINDOWS:
        cfg = W.CONFIGS[name]
        o = oracle_for(cfg)
        v, e, x = o.init_state()
        N = 2 * o.nv + o.ne
        t0 = time.time()
        total, dt, t = 0, 0.0, 0.0
        while time.time() - t0 < seconds and t < cfg["t_final"]:
            st, _, s_ = o.run(cfg["t_final"], v, e, x, t0=t, dt=dt, max_steps=1)
            if s_ != O.OK:
                break
            total += st["steps"]
            dt, t = st["dt"], st["t"]
        one = N * total / (time.time() - t0)
        del o
        pool = OraclePool([dict(cfg) for _ in range(nproc)], nproc, cfg["t_final"])
        try:
            steps_each = max(1, min(total, 20))
            upd, el = pool.advance(steps_each)
        finally:
            pool.close()
        out[name] = {"one_core": one, "all_cores": upd / el, "cores": pool.cores,
                     "steps_one_core": total, "steps_each_all_cores": steps_each}
    return out


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on the host cores, on the
    headline workload: each bench step advances the same seeded subset of
    sweep instances (2 per core, one spawned process per core) by 2 accepted
    RK2-average steps each."""
    world, rank, local = _dist()
    if rank != 0:
        return None
    import oracle as O
    O.lib()
    nproc = os.cpu_count() or 1
    sub = _cpu_subset(nproc)
    pool = OraclePool(sub, nproc, SWEEP_T_FINAL)
    chunk = 2
    try:
        for _ in range(args.warmup):
            pool.advance(chunk)
        upd, el = 0, 0.0
        for _ in range(args.steps):
            u, dt = pool.advance(chunk)
            upd += u
            el += dt
    finally:
        pool.close()
    value = upd / el
    sample = ("%d instances of the seeded sweep (the first 2 per core), %d accepted RK2-average "
              "steps each per bench step, %d spawned oracle processes" % (len(sub), chunk, pool.cores))
    return {"metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": SWEEP_WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": pool.cores,
                             "kind": "oracle", "sample": sample, "nproc": nproc},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-problem windows (2D blast 8x8, Taylor-Green 64x64, "
                         "3D blast 32^3, Gresho 256^2 Q3)")
    ap.add_argument("--full-runs", action="store_true",
                    help="also run every single-problem workload to its final time in FP64 "
                         "and mixed (several minutes)")
    ap.add_argument("--cpu-configs", action="store_true",
                    help="also time the oracle on each single-problem workload, one core and "
                         "all host cores")
    ap.add_argument("--quick", action="store_true",
                    help="the headline sweep only (no FP64 sweep, single-problem rates, "
                         "restricted force or full runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    line = run_reference(args) if args.impl == "reference" else run_native(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
