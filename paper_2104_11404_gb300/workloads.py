"""Seeded synthetic workloads shared by the tests, the smoke check and the
benchmark.  This module holds problem parameters and random-number recipes
only; none of the hydrodynamics arithmetic lives here, so both the CUDA path
and the CPU oracle can draw their inputs from it.

The named configurations reproduce the problem settings of Section 6.1 of
arXiv 2104.11404 (Sedov blast, Taylor-Green and Gresho vortices) on the mesh
sizes of the benchmark: they stand in for the paper's Laghos runs, which need
no external data.
"""
import math

import numpy as np

SEDOV, TAYLOR_GREEN, GRESHO, UNIFORM, TRIPLE_POINT = 1, 2, 3, 4, 5
RK2AVG, RK4 = 0, 1

CONFIGS = {
    # 2D point blast, [0,1]^2, 8x8 Q2/Q1, E0 = 0.25 in the origin element, t_f = 0.8
    "sedov2d_8": dict(dim=2, n=(8, 8, 1), order=2, problem=SEDOV, gamma=1.4,
                      lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1, blast_energy=0.25,
                      t_final=0.8),
    # 2D Taylor-Green vortex with its manufactured energy source, 64x64 Q2/Q1, t_f = 0.5,
    # CFL 0.1 as for the Taylor-Green runs of Table tab:fom
    "tg2d_64": dict(dim=2, n=(64, 64, 1), order=2, problem=TAYLOR_GREEN, gamma=5.0 / 3.0,
                    lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1, source=1, cfl=0.1,
                    t_final=0.5),
    # 3D point blast, [0,1]^3, 32^3 Q2/Q1, t_f = 0.6
    "sedov3d_32": dict(dim=3, n=(32, 32, 32), order=2, problem=SEDOV, gamma=1.4,
                       lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1, blast_energy=0.25,
                       t_final=0.6),
    # 2D Gresho vortex, [-0.5,0.5]^2, 256x256 Q3/Q2, no viscosity, t_f = 0.62
    "gresho2d_256": dict(dim=2, n=(256, 256, 1), order=3, problem=GRESHO, gamma=5.0 / 3.0,
                         lo=(-0.5, -0.5, 0.0), hi=(0.5, 0.5, 1.0), visc=0, t_final=0.62),
    # 3D triple point, [0,7] x [0,3] x [0,1.5], 28 x 12 x 4 Q2/Q1 (the mesh of Table
    # tab:fom, N_V = 38475, N_E = 10752), per-element rho0 / p / gamma, t_f = 0.8
    # (gamma here only satisfies the descriptor check; the problem sets its own)
    "triple3d_28": dict(dim=3, n=(28, 12, 4), order=2, problem=TRIPLE_POINT, gamma=1.5,
                        lo=(0.0, 0.0, 0.0), hi=(7.0, 3.0, 1.5), visc=1, t_final=0.8),
}

BATCH_SEED = 2104114040
BATCH_SIZES = (16, 24, 32, 48)


def scaled(name, n=None, t_final=None, **over):
    """A named configuration with another mesh size / final time / options."""
    cfg = dict(CONFIGS[name])
    if n is not None:
        cfg["n"] = tuple(n) + (1,) * (3 - len(n))
    if t_final is not None:
        cfg["t_final"] = t_final
    cfg.update(over)
    return cfg


def sizes(cfg):
    """(N_V, N_E, n_elements) of a configuration (dof counting of eq:fom)."""
    d, k = cfg["dim"], cfg["order"]
    n = cfg["n"][:d]
    nnodes = int(np.prod([m * k + 1 for m in n]))
    nel = int(np.prod(n))
    return d * nnodes, nel * k ** d, nel


def state_size(cfg):
    nv, ne, _ = sizes(cfg)
    return 2 * nv + ne


# ---- splitmix64 (Steele, Lea, Flood 2014) ------------------------------------

_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed):
        self.s = seed & _M64

    def next_u64(self):
        self.s = (self.s + 0x9E3779B97F4A7C15) & _M64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self):
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n):
        return int(self.uniform() * n)


def batch_instances(count=512, seed=BATCH_SEED):
    """Parameter sweep of point-blast instances: deposited energy U[0.1, 1.0],
    gamma U[1.3, 1.67], mesh n x n with n drawn from {16, 24, 32, 48}."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        e0 = 0.1 + 0.9 * rng.uniform()
        gam = 1.3 + 0.37 * rng.uniform()
        n = BATCH_SIZES[rng.below(len(BATCH_SIZES))]
        out.append(dict(dim=2, n=(n, n, 1), order=2, problem=SEDOV, gamma=gam,
                        lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1, blast_energy=e0,
                        t_final=0.8, index=i))
    return out


def element_sample(nelem, frac=0.05, seed=BATCH_SEED, stream=0):
    """ceil(frac * nelem) distinct element ids by a seeded Fisher-Yates
    shuffle, sorted (the sampled elements of a hyper-reduced evaluation)."""
    m = max(1, int(math.ceil(frac * nelem)))
    rng = SplitMix64(seed ^ ((stream + 1) * 0x9E3779B97F4A7C15))
    perm = list(range(nelem))
    for i in range(nelem - 1, 0, -1):
        j = rng.below(i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return np.array(sorted(perm[:m]), dtype=np.int32)


def perturbed_state(v, e, x, cfg, seed, vel=0.3, jitter=0.05, e_range=(0.5, 2.0)):
    """A random but valid state around (v, e, x): node jitter of `jitter`
    element widths / k, random velocities (zero on the walls is left to the
    caller's essential mask), random positive energies."""
    rng = np.random.default_rng(seed)
    d, k = cfg["dim"], cfg["order"]
    h = min((cfg["hi"][c] - cfg["lo"][c]) / cfg["n"][c] for c in range(d))
    x2 = x + (jitter / k) * h * rng.uniform(-1.0, 1.0, size=x.shape)
    v2 = vel * rng.normal(size=v.shape)
    e2 = rng.uniform(e_range[0], e_range[1], size=e.shape)
    return v2, e2, x2


def essential_mask(cfg):
    """Wall-normal velocity components (component c on faces x_c = lo, hi)."""
    d, k = cfg["dim"], cfg["order"]
    nn = [cfg["n"][c] * k + 1 for c in range(d)]
    idx = np.indices(nn[::-1]).reshape(d, -1)[::-1]
    mask = np.zeros((d, int(np.prod(nn))), dtype=bool)
    for c in range(d):
        mask[c] = (idx[c] == 0) | (idx[c] == nn[c] - 1)
    return mask.reshape(-1)
