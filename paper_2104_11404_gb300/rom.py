"""Convenience wrapper of the hyper-reduced online step (lh_rom_*) for Python
users: bases and offsets as torch tensors, reduced coordinates in and out.
All computation happens in liblagh.so."""
import torch

from . import lagh


class Rom:
    """Reduced model of a single-problem context (hydro.Hydro, FP64, no source
    term).  Phi_*: [rows, basis] column-major bases given as torch tensors of
    shape (basis, rows) (one basis vector per row of the tensor)."""

    def __init__(self, hydro, Phi_v, Phi_e, Phi_x, v_os, e_os, x_os, ns_f, ns_g,
                 samples_f=None, samples_g=None):
        dev = hydro.dev
        as_dev = lambda t: torch.as_tensor(t, dtype=torch.float64).to(dev).contiguous()
        self.Phi_v, self.Phi_e, self.Phi_x = as_dev(Phi_v), as_dev(Phi_e), as_dev(Phi_x)
        self.nbv, self.nbe, self.nbx = self.Phi_v.shape[0], self.Phi_e.shape[0], self.Phi_x.shape[0]
        self.hydro = hydro
        self.dev = dev
        self.r = lagh.lh_rom_create(hydro.ctx, self.Phi_v, self.nbv, self.Phi_e, self.nbe, self.Phi_x,
                                    self.nbx, as_dev(v_os), as_dev(e_os), as_dev(x_os), ns_f, ns_g,
                                    samples_f, samples_g)
        self.info, self.samples_f, self.samples_g, self.elements = lagh.lh_rom_info(self.r)

    def close(self):
        if getattr(self, "r", None):
            lagh.lh_rom_destroy(self.r)
            self.r = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, vh, eh, xh, t=0.0, dt=0.0):
        f = lambda a: torch.as_tensor(a, dtype=torch.float64).to(self.dev).contiguous()
        lagh.lh_rom_set_state(self.r, f(vh), f(eh), f(xh), t, dt)

    def get_state(self):
        z = lambda n: torch.zeros(n, dtype=torch.float64, device=self.dev)
        vh, eh, xh = z(self.nbv), z(self.nbe), z(self.nbx)
        t, dt = lagh.lh_rom_get_state(self.r, vh, eh, xh)
        return vh, eh, xh, t, dt

    def lift(self):
        v, e, x = self.hydro.zeros_v(), self.hydro.zeros_e(), self.hydro.zeros_v()
        lagh.lh_rom_lift(self.r, v, e, x)
        return v, e, x

    def step_fixed(self, dt):
        return lagh.lh_rom_step_fixed(self.r, dt)

    def run_to(self, t_final, max_steps=2 ** 62):
        return lagh.lh_rom_run_to(self.r, t_final, max_steps)
