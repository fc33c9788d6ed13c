"""Helpers that set up the CPU oracle and the CUDA library on the same seeded
workload for parity tests."""
import numpy as np

import oracle as O
from paper_2104_11404_gb300 import workloads as W


def oracle_for(cfg, **over):
    kw = dict(dim=cfg["dim"], nx=cfg["n"][0], ny=cfg["n"][1], nz=cfg["n"][2],
              lo=list(cfg["lo"]), hi=list(cfg["hi"]), order=cfg["order"],
              problem=cfg["problem"], gamma=cfg["gamma"], visc=cfg.get("visc", 1),
              blast_energy=cfg.get("blast_energy", 0.25), source=cfg.get("source", 1),
              e_uniform=cfg.get("e_uniform", 1.0), cfl=cfg.get("cfl", 0.5),
              integrator=cfg.get("integrator", 0))
    kw.update(over)
    return O.Oracle(**kw)


def gpu_for(cfg, precision="fp64", **kw):
    from paper_2104_11404_gb300.hydro import Hydro
    return Hydro(cfg, precision=precision, **kw)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def random_state(o, cfg, seed, **kw):
    v, e, x = o.init_state()
    v, e, x = W.perturbed_state(v, e, x, cfg, seed, **kw)
    v[W.essential_mask(cfg)] = 0.0
    return v, e, x


def rel_l2(a, b):
    """Relative L2 difference of eq:relerrors, ||a - b|| / ||a||."""
    na = np.linalg.norm(a)
    return np.linalg.norm(a - b) / (na if na > 0 else 1.0)


def max_rel(a, b):
    """Largest entry-wise difference relative to the largest reference entry."""
    m = np.abs(a).max()
    return np.abs(a - b).max() / (m if m > 0 else 1.0)
