"""Convenience wrapper of one library context for Python users: builds the
descriptors from a configuration dict (see workloads.CONFIGS) and moves
torch tensors through the C ABI.  All computation happens in liblagh.so."""
import torch

from . import lagh


def precision_id(precision):
    """The lh_precision of "fp64" or "mixed" (anything else is an error)."""
    ids = {"fp64": lagh.LH_FP64, "mixed": lagh.LH_MIXED}
    if precision not in ids:
        raise ValueError("precision must be 'fp64' or 'mixed', not %r" % (precision,))
    return ids[precision]


def descriptors(cfg, cg_rtol=None, cg_maxit=None, phys_overrides=None):
    """(mesh, disc, phys) descriptors of a configuration dict.  phys_overrides
    names fields of lh_phys_desc; an unknown name is an error (it would
    otherwise be a Python attribute that never reaches the library)."""
    L = lagh
    mesh = L.lh_mesh_desc()
    mesh.dim = cfg["dim"]
    mesh.nx, mesh.ny, mesh.nz = [int(v) for v in cfg["n"]]
    for i in range(3):
        mesh.lo[i] = float(cfg["lo"][i])
        mesh.hi[i] = float(cfg["hi"][i])
    disc = L.lh_disc_desc()
    disc.order = cfg["order"]
    disc.nq = cfg.get("nq", 2 * cfg["order"])
    phys = L.lh_default_phys()
    phys.problem = cfg["problem"]
    phys.gamma = float(cfg["gamma"])
    phys.visc = int(cfg.get("visc", 1))
    phys.source = int(cfg.get("source", 1))
    phys.blast_energy = float(cfg.get("blast_energy", 0.25))
    phys.e_uniform = float(cfg.get("e_uniform", 1.0))
    phys.cfl = float(cfg.get("cfl", 0.5))
    phys.integrator = int(cfg.get("integrator", 0))
    if cg_rtol is not None:
        phys.cg_rtol = cg_rtol
    if cg_maxit is not None:
        phys.cg_maxit = cg_maxit
    fields = {name for name, _ in L.lh_phys_desc._fields_}
    for k, v in (phys_overrides or {}).items():
        if k not in fields:
            raise KeyError("lh_phys_desc has no field %r" % (k,))
        setattr(phys, k, v)
    return mesh, disc, phys


class Hydro:
    def __init__(self, cfg, precision="fp64", stream=None, cg_rtol=None, cg_maxit=None,
                 phys_overrides=None):
        L = lagh
        self.cfg = dict(cfg)
        self.precision = precision_id(precision)
        mesh, disc, phys = descriptors(cfg, cg_rtol, cg_maxit, phys_overrides)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = L.lh_create(mesh, disc, phys, self.precision, self.stream.cuda_stream)
        self.layout = L.lh_layout(self.ctx)
        self.nv, self.ne = self.layout.nv, self.layout.ne
        self.nelem = self.layout.nelem
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "ctx", None):
            lagh.lh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros_v(self):
        return torch.zeros(self.nv, dtype=torch.float64, device=self.dev)

    def zeros_e(self):
        return torch.zeros(self.ne, dtype=torch.float64, device=self.dev)

    def init_state(self):
        lagh.lh_init_state(self.ctx)

    def set_state(self, v, e, x, t=0.0, dt=0.0):
        lagh.lh_set_state(self.ctx, v, e, x, t, dt)

    def get_state(self):
        v, e, x = self.zeros_v(), self.zeros_e(), self.zeros_v()
        t, dt = lagh.lh_get_state(self.ctx, v, e, x)
        return v, e, x, t, dt

    def force(self, v, e, x, vtest=None):
        F1 = self.zeros_v()
        FTv = self.zeros_e() if vtest is not None else None
        dt = lagh.lh_force(self.ctx, v, e, x, F1, vtest, FTv)
        return F1, FTv, dt

    def force_sampled(self, elem_ids, v, e, x, vtest=None):
        n = int(elem_ids.numel())
        d, nd1, nd2 = self.layout.dim, self.layout.ndof_h1, self.layout.ndof_l2
        F1 = torch.zeros(n * d * nd1, dtype=torch.float64, device=self.dev)
        FTv = torch.zeros(n * nd2, dtype=torch.float64, device=self.dev) if vtest is not None else None
        dt = lagh.lh_force_sampled(self.ctx, elem_ids, n, v, e, x, F1, vtest, FTv)
        return F1, FTv, dt

    def mass_apply_v(self, a):
        out = self.zeros_v()
        lagh.lh_mass_apply_v(self.ctx, a, out)
        return out

    def mass_solve_v(self, rhs):
        out = self.zeros_v()
        its, rr = lagh.lh_mass_solve_v(self.ctx, rhs, out)
        return out, its, rr

    def mass_solve_e(self, rhs):
        out = self.zeros_e()
        lagh.lh_mass_solve_e(self.ctx, rhs, out)
        return out

    def total_energy(self):
        return lagh.lh_total_energy(self.ctx)

    def step_fixed(self, dt):
        return lagh.lh_step_fixed(self.ctx, dt)

    def step(self, t_final):
        return lagh.lh_step(self.ctx, t_final)

    def run_to(self, t_final, max_steps=2 ** 62, dt_log=None):
        cap = int(dt_log.numel()) if dt_log is not None else 0
        return lagh.lh_run_to(self.ctx, t_final, max_steps, dt_log, cap)
