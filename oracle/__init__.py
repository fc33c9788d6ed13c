"""Python access to the plain FP64 CPU oracle (oracle/lagh_oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the correctness reference for the
CUDA library: the tests, the smoke check and the CPU-baseline leg of the
benchmark use it; the product path never does.  It follows the semi-discrete
system of eq:fom, the RK2-average scheme of eq:RK2-avg (or RK4, eq:RK4) and the step control
of Section 2.2.3 of arXiv 2104.11404; the readings of what the paper leaves open
are listed at the top of lagh_oracle.c.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SEDOV, TAYLOR_GREEN, GRESHO, UNIFORM, TRIPLE_POINT = 1, 2, 3, 4, 5
RK2AVG, RK4 = 0, 1
OK, EINVAL, ETANGLED, ENONFINITE, EDTMIN, ECG = 0, 1, 4, 5, 6, 7

_dp = ctypes.POINTER(ctypes.c_double)


class _Config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("order", ctypes.c_int), ("nq", ctypes.c_int), ("problem", ctypes.c_int),
        ("gamma", ctypes.c_double), ("blast_energy", ctypes.c_double),
        ("e_uniform", ctypes.c_double), ("visc", ctypes.c_int),
        ("cfl", ctypes.c_double), ("cfl_mu", ctypes.c_double),
        ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("gamma_dt", ctypes.c_double),
        ("cg_rtol", ctypes.c_double), ("cg_maxit", ctypes.c_int),
        ("dt_min_frac", ctypes.c_double), ("q1", ctypes.c_double), ("q2", ctypes.c_double),
        ("source", ctypes.c_int), ("integrator", ctypes.c_int),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_long), ("rejects", ctypes.c_long), ("cg_iters", ctypes.c_long),
                ("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("energy0", ctypes.c_double), ("energy", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.lho_create.restype = ctypes.c_void_p
        L.lho_create.argtypes = [ctypes.POINTER(_Config)]
        L.lho_destroy.argtypes = [ctypes.c_void_p]
        L.lho_default_config.argtypes = [ctypes.POINTER(_Config)]
        L.lho_sizes.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_long)] * 5
        L.lho_local_sizes.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 3
        L.lho_init_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.lho_force.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.lho_element_force_matrix.argtypes = [ctypes.c_void_p, ctypes.c_long, _dp, _dp, _dp, _dp]
        L.lho_energy_source.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.lho_mass_apply_v.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.lho_mass_solve_v.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.POINTER(ctypes.c_int), _dp]
        L.lho_mass_solve_v_dense.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.lho_mass_apply_e.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.lho_mass_solve_e.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.lho_step.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp, _dp, _dp,
                               ctypes.POINTER(ctypes.c_long)]
        L.lho_step_rk4.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp, _dp, _dp,
                                   ctypes.POINTER(ctypes.c_long)]
        L.lho_run_snapshots.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_long, _dp, _dp, _dp, _dp, ctypes.POINTER(_Stats),
                                        _dp, _dp, _dp, ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
        L.lho_svd_jacobi.argtypes = [ctypes.c_long, ctypes.c_long, _dp, _dp, ctypes.c_double,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.lho_pod.argtypes = [ctypes.c_long, ctypes.c_long, _dp, _dp, ctypes.c_double, _dp, _dp,
                              ctypes.POINTER(ctypes.c_long)]
        L.lho_estimate_elements.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, _dp,
                                            _dp, _dp, ctypes.POINTER(ctypes.c_double)]
        L.lho_run.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                              _dp, _dp, _dp, _dp, ctypes.POINTER(_Stats), _dp, ctypes.c_long]
        L.lho_total_energy.restype = ctypes.c_double
        L.lho_total_energy.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.lho_gauss_lobatto.argtypes = [ctypes.c_int, _dp]
        L.lho_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
        L.lho_lagrange.argtypes = [ctypes.c_int, _dp, ctypes.c_double, _dp, _dp]
        L.lho_qpoint.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                 _dp, _dp, _dp]
        L.lho_sym_min_eig.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def default_config():
    c = _Config()
    lib().lho_default_config(ctypes.byref(c))
    return c


class Oracle:
    """One problem instance on a Cartesian box mesh (see lagh_oracle.h)."""

    def __init__(self, **kw):
        c = default_config()
        if "dim" in kw and "nq" not in kw and "order" in kw:
            pass
        for key, val in kw.items():
            if key in ("lo", "hi"):
                arr = getattr(c, key)
                for i, x in enumerate(val):
                    arr[i] = float(x)
            else:
                setattr(c, key, val)
        if "nq" not in kw:
            c.nq = 2 * c.order
        self.cfg = c
        self._h = lib().lho_create(ctypes.byref(c))
        if not self._h:
            raise ValueError("invalid oracle configuration")
        vals = [ctypes.c_long() for _ in range(5)]
        lib().lho_sizes(self._h, *[ctypes.byref(v) for v in vals])
        self.nv, self.ne, self.nqp, self.nelem, self.nnodes = [v.value for v in vals]
        loc = [ctypes.c_int() for _ in range(3)]
        lib().lho_local_sizes(self._h, *[ctypes.byref(v) for v in loc])
        self.nd1, self.nd2, self.nqe = [v.value for v in loc]
        self.dim = c.dim

    def __del__(self):
        if getattr(self, "_h", None):
            lib().lho_destroy(self._h)
            self._h = None

    # state ---------------------------------------------------------------
    def init_state(self):
        v = np.zeros(self.nv)
        e = np.zeros(self.ne)
        x = np.zeros(self.nv)
        lib().lho_init_state(self._h, _p(v), _p(e), _p(x))
        return v, e, x

    # force ---------------------------------------------------------------
    def force(self, v, e, x, vtest=None):
        F1 = np.zeros(self.nv)
        FTv = np.zeros(self.ne) if vtest is not None else None
        dt = ctypes.c_double()
        st = lib().lho_force(self._h, _p(v), _p(e), _p(x), _p(vtest), _p(F1), _p(FTv),
                             ctypes.byref(dt))
        return F1, FTv, dt.value, st

    def element_force_matrix(self, elem, v, e, x):
        FK = np.zeros((self.dim * self.nd1, self.nd2))
        st = lib().lho_element_force_matrix(self._h, elem, _p(v), _p(e), _p(x), _p(FK))
        if st not in (OK,):
            raise RuntimeError("element force status %d" % st)
        return FK

    def estimate_elements(self, elems, v, e, x):
        """Estimate of eq:adaptive-timestep over the listed elements only."""
        ids = np.ascontiguousarray(elems, dtype=np.int64)
        tau = ctypes.c_double()
        st = lib().lho_estimate_elements(self._h, ids.ctypes.data, len(ids), _p(v), _p(e), _p(x),
                                         ctypes.byref(tau))
        return tau.value, st

    def energy_source(self, x):
        s = np.zeros(self.ne)
        lib().lho_energy_source(self._h, _p(x), _p(s))
        return s

    # mass ----------------------------------------------------------------
    def mass_apply_v(self, a):
        out = np.zeros(self.nv)
        lib().lho_mass_apply_v(self._h, _p(np.ascontiguousarray(a, dtype=np.float64)), _p(out))
        return out

    def mass_solve_v(self, rhs):
        out = np.zeros(self.nv)
        it = ctypes.c_int()
        rr = ctypes.c_double()
        st = lib().lho_mass_solve_v(self._h, _p(np.ascontiguousarray(rhs, dtype=np.float64)),
                                    _p(out), ctypes.byref(it), ctypes.byref(rr))
        return out, it.value, rr.value, st

    def mass_solve_v_dense(self, rhs):
        out = np.zeros(self.nv)
        st = lib().lho_mass_solve_v_dense(self._h, _p(np.ascontiguousarray(rhs, dtype=np.float64)),
                                          _p(out))
        if st != OK:
            raise RuntimeError("dense solve status %d" % st)
        return out

    def mass_apply_e(self, a):
        out = np.zeros(self.ne)
        lib().lho_mass_apply_e(self._h, _p(np.ascontiguousarray(a, dtype=np.float64)), _p(out))
        return out

    def mass_solve_e(self, rhs):
        out = np.zeros(self.ne)
        lib().lho_mass_solve_e(self._h, _p(np.ascontiguousarray(rhs, dtype=np.float64)), _p(out))
        return out

    # time integration ----------------------------------------------------
    def step(self, dt, v, e, x):
        """One RK2-average step in place; returns (tau, cg_iters, status)."""
        tau = ctypes.c_double()
        its = ctypes.c_long()
        st = lib().lho_step(self._h, float(dt), _p(v), _p(e), _p(x), ctypes.byref(tau),
                            ctypes.byref(its))
        return tau.value, its.value, st

    def step_rk4(self, dt, v, e, x):
        """One RK4 step in place; returns (tau, cg_iters, status)."""
        tau = ctypes.c_double()
        its = ctypes.c_long()
        st = lib().lho_step_rk4(self._h, float(dt), _p(v), _p(e), _p(x), ctypes.byref(tau),
                                ctypes.byref(its))
        return tau.value, its.value, st

    def run(self, t_final, v, e, x, t0=0.0, dt=0.0, max_steps=10 ** 9, log_cap=100000):
        """Step control loop in place; returns (stats dict, accepted dt list, status)."""
        dtc = ctypes.c_double(dt)
        stats = _Stats()
        log = np.zeros(log_cap)
        st = lib().lho_run(self._h, float(t0), float(t_final), int(max_steps), _p(v), _p(e),
                           _p(x), ctypes.byref(dtc), ctypes.byref(stats), _p(log), log_cap)
        d = {k: getattr(stats, k) for k, _ in _Stats._fields_}
        return d, log[:min(stats.steps, log_cap)].copy(), st

    def run_snapshots(self, t_final, v, e, x, cap, t0=0.0, dt=0.0, max_steps=10 ** 9):
        """lho_run collecting the RK2-average stage snapshots (S^{n+1/2} and
        S^{n+1} of every accepted step); returns (stats, Sv, Se, Sx, status)
        with the snapshot matrices as [column, row] arrays."""
        dtc = ctypes.c_double(dt)
        stats = _Stats()
        Sv = np.zeros((cap, self.nv))
        Se = np.zeros((cap, self.ne))
        Sx = np.zeros((cap, self.nv))
        cnt = ctypes.c_long()
        st = lib().lho_run_snapshots(self._h, float(t0), float(t_final), int(max_steps), _p(v),
                                     _p(e), _p(x), ctypes.byref(dtc), ctypes.byref(stats), _p(Sv),
                                     _p(Se), _p(Sx), cap, ctypes.byref(cnt))
        d = {k: getattr(stats, k) for k, _ in _Stats._fields_}
        n = min(cnt.value, cap)
        d["snapshots"] = cnt.value
        return d, Sv[:n], Se[:n], Sx[:n], st

    def total_energy(self, v, e):
        return lib().lho_total_energy(self._h, _p(v), _p(e))

    def qpoint(self, J, gradv_ref, e_q, rho0detJ0):
        d = self.dim
        J = np.ascontiguousarray(J, dtype=np.float64).reshape(d * d)
        G = np.ascontiguousarray(gradv_ref, dtype=np.float64).reshape(d * d)
        sigma = np.zeros(d * d)
        tau = ctypes.c_double()
        mu = ctypes.c_double()
        st = lib().lho_qpoint(self._h, _p(J), _p(G), float(e_q), float(rho0detJ0), _p(sigma),
                              ctypes.byref(tau), ctypes.byref(mu))
        return sigma.reshape(d, d), tau.value, mu.value, st

    def essential_mask(self):
        """Boolean mask of the essential (wall-normal) velocity components."""
        d = self.dim
        nn = [self.cfg.nx * self.cfg.order + 1, self.cfg.ny * self.cfg.order + 1,
              self.cfg.nz * self.cfg.order + 1][:d]
        idx = np.indices(nn[::-1]).reshape(d, -1)[::-1]  # idx[c] = node index along c
        mask = np.zeros((d, int(np.prod(nn))), dtype=bool)
        for c in range(d):
            mask[c] = (idx[c] == 0) | (idx[c] == nn[c] - 1)
        return mask.reshape(-1)


def gauss_lobatto(n):
    x = np.zeros(n)
    lib().lho_gauss_lobatto(n, _p(x))
    return x


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().lho_gauss_legendre(n, _p(x), _p(w))
    return x, w


def lagrange(nodes, t):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    n = len(nodes)
    val = np.zeros(n)
    der = np.zeros(n)
    lib().lho_lagrange(n, _p(nodes), float(t), _p(val), _p(der))
    return val, der


def sym_min_eig(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    d = A.shape[0]
    lam = ctypes.c_double()
    s = np.zeros(d)
    lib().lho_sym_min_eig(d, _p(A.reshape(-1)), ctypes.byref(lam), _p(s))
    return lam.value, s


def svd_jacobi(A, tol=1e-15, max_sweeps=60):
    """One-sided Jacobi thin SVD of A (rows x cols); returns (U Sigma columns as
    an array [col, row], sigma, sweeps, status)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)   # column-major storage
    n, m = A.shape
    sg = np.zeros(n)
    sw = ctypes.c_int()
    st = lib().lho_svd_jacobi(m, n, _p(A), _p(sg), tol, max_sweeps, ctypes.byref(sw))
    return A, sg, sw.value, st


def pod(S_cols, offset=None, eps=0.9999):
    """POD of snapshots given as an array [column, row]: returns (U as
    [column, row] in descending singular-value order, sigma, k, status)."""
    S = np.ascontiguousarray(S_cols, dtype=np.float64)
    n, m = S.shape
    U = np.zeros((n, m))
    sg = np.zeros(n)
    k = ctypes.c_long()
    off = None if offset is None else np.ascontiguousarray(offset, dtype=np.float64)
    st = lib().lho_pod(m, n, _p(S), _p(off), eps, _p(U), _p(sg), ctypes.byref(k))
    return U, sg, k.value, st
