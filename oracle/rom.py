"""Plain reference of the hyper-reduced online step of Section 3 with the
SNS bases of Section 4.2 and DEIM sampling of Section 4.3.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): numpy on top of the C
oracle's force and mass routines; the product path never imports it.

Every operation is written at full order and then restricted, so it checks the
GPU's sampled-element computation against the definition:
  * SNS bases (eq:rom-hr-sns): Phi_F = M_V Phi_v with the essential rows set to
    zero (F.1 has zero essential components, reading R15), Phi_G = M_E Phi_e;
  * DEIM sampling with over-sampling (reading R16): basis vector j receives
    its share of the ns samples, each at the largest entry of the residual of
    its gappy least-squares reconstruction from the basis vectors before it
    (for ns = m this is the greedy DEIM of the paper's Algorithm 1 reference);
  * the least-squares coefficients of eq:sol-ls-hyper, P = (Z^T Phi)^+;
  * the RK2-average hyper-reduced step of eq:RK2-avg-rom-hr: the lifted state
    (eq:discretesolrepresentation) is formed at full order, F.1 and F^T w are
    the full-order force of the oracle sampled at Z, and the time-step
    estimate is the minimum over the elements that touch a sampled entry
    (reading R17: the lifting exists only there).
"""
import numpy as np

from . import Oracle  # noqa: F401  (type of the problem object)


def sns_bases(o, Phi_v, Phi_e):
    """Phi_F = M_V^0 Phi_v (essential rows zero) and Phi_G = M_E Phi_e;
    bases as arrays [row, column]."""
    ess = o.essential_mask()
    PF = np.stack([o.mass_apply_v(Phi_v[:, j]) for j in range(Phi_v.shape[1])], axis=1)
    PF[ess, :] = 0.0
    PG = np.stack([o.mass_apply_e(Phi_e[:, j]) for j in range(Phi_e.shape[1])], axis=1)
    return PF, PG


def deim(Phi, ns):
    """Sample rows of Phi (N x m) by greedy DEIM with over-sampling to ns >= m
    rows (reading R16); ties go to the lowest row index."""
    N, m = Phi.shape
    if not (m <= ns <= N):
        raise ValueError("need m <= ns <= N")
    p = []
    for j in range(m):
        share = ns // m + (1 if j < ns % m else 0)
        for _ in range(share):
            if j == 0:
                r = Phi[:, 0].copy()
            else:
                c = np.linalg.lstsq(Phi[p, :j], Phi[p, j], rcond=None)[0]
                r = Phi[:, j] - Phi[:, :j] @ c
            r = np.abs(r)
            r[p] = -1.0
            p.append(int(np.argmax(r)))
    return np.array(p, dtype=np.int64)


def element_nodes(o, el):
    """Global nodes of element el (lexicographic layout, x fastest)."""
    d, k = o.dim, o.cfg.order
    n = [o.cfg.nx, o.cfg.ny, o.cfg.nz][:d]
    nn = [m * k + 1 for m in n]
    E, r = [], el
    for c in range(d):
        E.append(r % n[c])
        r //= n[c]
    out = []
    for i in range((k + 1) ** d):
        a = [(i // (k + 1) ** c) % (k + 1) for c in range(d)]
        idx = 0
        for c in reversed(range(d)):
            idx = idx * nn[c] + E[c] * k + a[c]
        out.append(idx)
    return out


def sampled_elements(o, pF, pG):
    """Elements whose force the hyper-reduced step evaluates: every element
    touching a node of a sampled F.1 entry, and the element of every sampled
    F^T w entry (sorted)."""
    nodes = set(int(i) % o.nnodes for i in pF)
    els = set(int(j) // o.nd2 for j in pG)
    for el in range(o.nelem):
        if nodes.intersection(element_nodes(o, el)):
            els.add(el)
    return np.array(sorted(els), dtype=np.int64)


class RomOracle:
    """Hyper-reduced RK2-average ROM (eq:RK2-avg-rom-hr) with SNS bases."""

    def __init__(self, o, Phi_v, Phi_e, Phi_x, v_os, e_os, x_os, pF, pG):
        self.o = o
        self.Phi_v, self.Phi_e, self.Phi_x = Phi_v, Phi_e, Phi_x
        self.v_os, self.e_os, self.x_os = v_os, e_os, x_os
        self.PF, self.PG = sns_bases(o, Phi_v, Phi_e)
        self.pF, self.pG = np.asarray(pF), np.asarray(pG)
        self.AF = np.linalg.pinv(self.PF[self.pF, :])       # (Z^T Phi_F)^+
        self.AG = np.linalg.pinv(self.PG[self.pG, :])
        self.els = sampled_elements(o, self.pF, self.pG)

    def lift(self, vh, eh, xh):
        return (self.v_os + self.Phi_v @ vh, self.e_os + self.Phi_e @ eh,
                self.x_os + self.Phi_x @ xh)

    def _f(self, v, e, x):
        F1, _, _, st = self.o.force(v, e, x)
        assert st == 0
        tau, _ = self.o.estimate_elements(self.els, v, e, x)
        return self.AF @ F1[self.pF], tau

    def _g(self, v, e, x, w):
        _, FTw, _, st = self.o.force(v, e, x, vtest=w)
        assert st == 0
        return self.AG @ FTw[self.pG]

    def step(self, dt, vh, eh, xh):
        """One step of eq:RK2-avg-rom-hr; returns the new coordinates and the
        estimate (minimum over both stages)."""
        v, e, x = self.lift(vh, eh, xh)
        f, tau1 = self._f(v, e, x)
        vh_half = vh - 0.5 * dt * f
        w = self.v_os + self.Phi_v @ vh_half
        eh_half = eh + 0.5 * dt * self._g(v, e, x, w)
        xh_half = xh + 0.5 * dt * (self.Phi_x.T @ w)
        v2, e2, x2 = self.lift(vh_half, eh_half, xh_half)
        f2, tau2 = self._f(v2, e2, x2)
        vh_new = vh - dt * f2
        vbar = 0.5 * (vh + vh_new)
        wbar = self.v_os + self.Phi_v @ vbar
        eh_new = eh + dt * self._g(v2, e2, x2, wbar)
        xh_new = xh + dt * (self.Phi_x.T @ wbar)
        return vh_new, eh_new, xh_new, min(tau1, tau2)

    def run(self, t_final, vh, eh, xh, dt=0.0, t0=0.0, max_steps=10 ** 9):
        """The step control of Section 2.2.3 on the hyper-reduced step (the
        FOM rules, the estimate of reading R17); returns (coordinates, t, dt,
        steps, rejects, accepted step sizes)."""
        c = self.o.cfg
        t = t0
        if not dt > 0.0:
            v, e, x = self.lift(vh, eh, xh)
            dt, _ = self.o.estimate_elements(self.els, v, e, x)
        steps = rejects = 0
        log = []
        while t < t_final and steps < max_steps:
            dt_use, last = dt, False
            if t + dt_use >= t_final:
                dt_use, last = t_final - t, True
            a, b, cc, tau = self.step(dt_use, vh, eh, xh)
            if dt_use >= tau:
                dt = c.beta1 * dt_use
                rejects += 1
                if dt < c.dt_min_frac * t_final:
                    raise RuntimeError("time step collapsed")
                continue
            vh, eh, xh = a, b, cc
            steps += 1
            log.append(dt_use)
            t = t_final if last else t + dt_use
            dt = c.beta2 * dt_use if dt_use <= c.gamma_dt * tau else dt_use
        return vh, eh, xh, t, dt, steps, rejects, np.array(log)
