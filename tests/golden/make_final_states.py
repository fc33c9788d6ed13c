"""Writes the oracle's final states used by tests/test_gpu_finaltime.py.

Calls only the CPU oracle (oracle/) on the problems of Section 6.1 at the
sizes of Table tab:fom where the oracle finishes in minutes (3D blast 8^3
Q2/Q1 to t = 0.6, Gresho 32^2 Q3/Q2 to t = 0.62) and on the 64x64 2D
Taylor-Green benchmark configuration to t = 0.5, each from its initial
condition under the step control of Section 2.2.3.  One spawned process per
problem.  Output: tests/golden/final_<name>.npz with the final v, e, x, the
accepted step sizes in order, the step and reject counts and the total energy
before and after.

    python tests/golden/make_final_states.py [name ...]
"""
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

PROBLEMS = {
    # name: (configuration, mesh)
    "tg2d_64": ("tg2d_64", (64, 64)),
    "sedov3d_8": ("sedov3d_32", (8, 8, 8)),
    "gresho2d_32": ("gresho2d_256", (32, 32)),
}


def run(name):
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_2104_11404_gb300 import workloads as W
    from tests._pair import oracle_for
    base, n = PROBLEMS[name]
    cfg = W.scaled(base, n=n)
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    t0 = time.time()
    stats, log, st = o.run(cfg["t_final"], v, e, x, log_cap=200000)
    if st != 0:
        raise RuntimeError("%s: oracle status %d" % (name, st))
    np.savez_compressed(os.path.join(HERE, "final_%s.npz" % name), v=v, e=e, x=x, dt_log=log,
                        steps=stats["steps"], rejects=stats["rejects"],
                        energy0=stats["energy0"], energy=stats["energy"], t_final=stats["t"])
    return name, stats["steps"], stats["rejects"], time.time() - t0


if __name__ == "__main__":
    names = sys.argv[1:] or list(PROBLEMS)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(names)) as pool:
        for res in pool.imap_unordered(run, names):
            print("%s: %d steps, %d rejects, %.0f s" % res, flush=True)
