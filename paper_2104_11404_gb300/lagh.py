"""Thin Python binding of the C ABI in include/lagh.h (argument marshalling only).

Every numerical step runs in the CUDA library _lib/liblagh.so; this module only
converts descriptors, passes device pointers of torch tensors (or host
pointers where the ABI allows them) and turns status codes into exceptions.
Importing it does not need a GPU; creating a context does.  There is no
fallback: if the library is missing the calls raise.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "liblagh.so")

LH_OK, LH_EINVAL, LH_ENOMEM, LH_ECUDA, LH_ETANGLED, LH_ENONFINITE, LH_EDTMIN, LH_ECG, \
    LH_ETIMEOUT, LH_EUNSUPPORTED, LH_ETOOLARGE = range(11)
LH_FP64, LH_MIXED = 0, 1
LH_SEDOV, LH_TAYLOR_GREEN, LH_GRESHO, LH_UNIFORM, LH_TRIPLE_POINT = 1, 2, 3, 4, 5
LH_RK2AVG, LH_RK4 = 0, 1
LH_PRECOND_JACOBI, LH_PRECOND_TENSOR, LH_PRECOND_EXACT, LH_PRECOND_TENSOR64, LH_PRECOND_AUTO = \
    0, 1, 2, 3, 4

# every entry point declared in include/lagh.h
API_NAMES = [
    "lh_default_phys", "lh_status_string", "lh_create", "lh_destroy", "lh_last_error",
    "lh_layout", "lh_init_state", "lh_set_state", "lh_get_state", "lh_force",
    "lh_force_sampled", "lh_mass_apply_v", "lh_mass_solve_v", "lh_mass_solve_e",
    "lh_total_energy", "lh_step_fixed", "lh_step", "lh_run_to", "lh_force_static",
    "lh_precond_apply", "lh_batch_create", "lh_batch_destroy", "lh_batch_last_error",
    "lh_batch_layout", "lh_batch_init_state", "lh_batch_set_state", "lh_batch_get_state",
    "lh_batch_query", "lh_batch_run_to", "lh_batch_step_fixed", "lh_batch_total_energy",
    "lh_batch_force_sampled", "lh_batch_autotune", "lh_batch_tuning_get",
    "lh_check_conversions", "lh_peak_probe", "lh_peak_probe_lanes", "lh_pod", "lh_batch_snapshots",
    "lh_batch_snapshot_count", "lh_rom_create", "lh_rom_destroy", "lh_rom_last_error",
    "lh_rom_info", "lh_rom_set_state", "lh_rom_get_state", "lh_rom_lift", "lh_rom_step_fixed",
    "lh_rom_run_to",
]


class lh_mesh_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class lh_disc_desc(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("nq", ctypes.c_int32)]


class lh_phys_desc(ctypes.Structure):
    _fields_ = [("problem", ctypes.c_int32), ("visc", ctypes.c_int32), ("source", ctypes.c_int32),
                ("cg_maxit", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("blast_energy", ctypes.c_double), ("e_uniform", ctypes.c_double),
                ("cfl", ctypes.c_double), ("cfl_mu", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("gamma_dt", ctypes.c_double), ("q1", ctypes.c_double), ("q2", ctypes.c_double),
                ("cg_rtol", ctypes.c_double), ("dt_min_frac", ctypes.c_double),
                ("cg_precond", ctypes.c_int32), ("direct_launch", ctypes.c_int32),
                ("cg_cluster", ctypes.c_int32), ("cg_tiles", ctypes.c_int32),
                ("integrator", ctypes.c_int32)]


class lh_layout_info(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("ne", ctypes.c_int64), ("nqp", ctypes.c_int64),
                ("nelem", ctypes.c_int64), ("nnodes", ctypes.c_int64),
                ("dim", ctypes.c_int32), ("order", ctypes.c_int32), ("nq", ctypes.c_int32),
                ("ndof_h1", ctypes.c_int32), ("ndof_l2", ctypes.c_int32), ("nqe", ctypes.c_int32),
                ("nodes_per_dim", ctypes.c_int32 * 3), ("precision", ctypes.c_int32),
                ("n_essential", ctypes.c_int64), ("precond_kernels", ctypes.c_int32)]


class lh_run_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("rejects", ctypes.c_int64),
                ("cg_iters", ctypes.c_int64), ("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("energy0", ctypes.c_double), ("energy", ctypes.c_double),
                ("wall_ms", ctypes.c_double)]


class lh_batch_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("rejects", ctypes.c_int64),
                ("cg_iters", ctypes.c_int64), ("attempts", ctypes.c_int64),
                ("instances_done", ctypes.c_int64), ("dof_updates", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("wall_ms", ctypes.c_double)]


class lh_rom_info_t(ctypes.Structure):
    _fields_ = [("nb_v", ctypes.c_int32), ("nb_e", ctypes.c_int32), ("nb_x", ctypes.c_int32),
                ("ns_f", ctypes.c_int32), ("ns_g", ctypes.c_int32), ("n_elems", ctypes.c_int64),
                ("n_rows_v", ctypes.c_int64), ("n_rows_e", ctypes.c_int64)]


class lh_batch_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("smem_lines", ctypes.c_int32), ("qpt", ctypes.c_int32)]


_vp = ctypes.c_void_p
_dp = ctypes.c_void_p  # device or host double*, passed as an address
_lib = None


def load():
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblagh.so is not built: run paper_2104_11404_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    S = ctypes.c_int
    L.lh_default_phys.argtypes = [ctypes.POINTER(lh_phys_desc)]
    L.lh_default_phys.restype = None
    L.lh_status_string.argtypes = [S]
    L.lh_status_string.restype = ctypes.c_char_p
    L.lh_create.argtypes = [ctypes.POINTER(lh_mesh_desc), ctypes.POINTER(lh_disc_desc),
                            ctypes.POINTER(lh_phys_desc), ctypes.c_int32, _vp,
                            ctypes.POINTER(_vp)]
    L.lh_destroy.argtypes = [_vp]
    L.lh_last_error.argtypes = [_vp]
    L.lh_last_error.restype = ctypes.c_char_p
    L.lh_layout.argtypes = [_vp, ctypes.POINTER(lh_layout_info)]
    L.lh_init_state.argtypes = [_vp]
    L.lh_set_state.argtypes = [_vp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double]
    L.lh_get_state.argtypes = [_vp, _dp, _dp, _dp, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]
    L.lh_force.argtypes = [_vp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.POINTER(ctypes.c_double)]
    L.lh_force_sampled.argtypes = [_vp, _vp, ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp,
                                   ctypes.POINTER(ctypes.c_double)]
    L.lh_mass_apply_v.argtypes = [_vp, _dp, _dp]
    L.lh_mass_solve_v.argtypes = [_vp, _dp, _dp, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_double)]
    L.lh_mass_solve_e.argtypes = [_vp, _dp, _dp]
    L.lh_precond_apply.argtypes = [_vp, _dp, _dp]
    L.lh_total_energy.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    L.lh_step_fixed.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.lh_step.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.lh_run_to.argtypes = [_vp, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(lh_run_stats),
                            _dp, ctypes.c_int64]
    L.lh_force_static.argtypes = [ctypes.POINTER(lh_mesh_desc), ctypes.POINTER(lh_disc_desc),
                                  ctypes.POINTER(lh_phys_desc), _dp, _dp, _dp, _dp,
                                  ctypes.POINTER(ctypes.c_double), _vp]
    P = ctypes.POINTER
    L.lh_batch_create.argtypes = [ctypes.c_int32, P(lh_mesh_desc), P(lh_disc_desc),
                                  P(lh_phys_desc), ctypes.c_int32, _vp, P(lh_batch_tuning),
                                  P(_vp)]
    L.lh_batch_destroy.argtypes = [_vp]
    L.lh_batch_last_error.argtypes = [_vp]
    L.lh_batch_last_error.restype = ctypes.c_char_p
    L.lh_batch_layout.argtypes = [_vp, _vp, _vp, _vp]
    L.lh_batch_init_state.argtypes = [_vp]
    L.lh_batch_set_state.argtypes = [_vp, _dp, _dp, _dp, _dp, _dp]
    L.lh_batch_get_state.argtypes = [_vp, _dp, _dp, _dp]
    L.lh_batch_query.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.lh_batch_run_to.argtypes = [_vp, ctypes.c_double, ctypes.c_int64, P(lh_batch_stats)]
    L.lh_batch_step_fixed.argtypes = [_vp, _dp, P(lh_batch_stats)]
    L.lh_batch_total_energy.argtypes = [_vp, _dp]
    L.lh_batch_force_sampled.argtypes = [_vp, _vp, _vp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.lh_batch_autotune.argtypes = [_vp, ctypes.c_int32, P(lh_batch_tuning)]
    L.lh_batch_tuning_get.argtypes = [_vp, P(lh_batch_tuning)]
    L.lh_check_conversions.argtypes = [_dp, ctypes.c_int64, _vp, _dp, _dp, _vp]
    L.lh_pod.argtypes = [_dp, ctypes.c_int64, ctypes.c_int64, _dp, ctypes.c_double, _dp, _dp, _dp,
                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), _vp]
    L.lh_batch_snapshots.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.c_int64, _dp, _dp, _dp]
    L.lh_batch_snapshot_count.argtypes = [_vp, _vp]
    L.lh_rom_create.argtypes = [_vp, _dp, ctypes.c_int32, _dp, ctypes.c_int32, _dp, ctypes.c_int32,
                                _dp, _dp, _dp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, P(_vp)]
    L.lh_rom_destroy.argtypes = [_vp]
    L.lh_rom_last_error.argtypes = [_vp]
    L.lh_rom_last_error.restype = ctypes.c_char_p
    L.lh_rom_info.argtypes = [_vp, P(lh_rom_info_t), _vp, _vp, _vp]
    L.lh_rom_set_state.argtypes = [_vp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double]
    L.lh_rom_get_state.argtypes = [_vp, _dp, _dp, _dp, P(ctypes.c_double), P(ctypes.c_double)]
    L.lh_rom_lift.argtypes = [_vp, _dp, _dp, _dp]
    L.lh_rom_step_fixed.argtypes = [_vp, ctypes.c_double, P(ctypes.c_double)]
    L.lh_rom_run_to.argtypes = [_vp, ctypes.c_double, ctypes.c_int64, P(lh_run_stats)]
    L.lh_peak_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, _vp, _vp,
                                ctypes.POINTER(ctypes.c_double)]
    L.lh_peak_probe_lanes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _vp, _vp,
                                      ctypes.POINTER(ctypes.c_double)]
    for name in API_NAMES:
        if name not in ("lh_default_phys", "lh_status_string", "lh_last_error",
                        "lh_batch_last_error", "lh_rom_last_error"):
            getattr(L, name).restype = S
    _lib = L
    return L


class LaghError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (status_string(status), status, msg))
        self.status = status


def status_string(s):
    return load().lh_status_string(s).decode()


def _ptr(t):
    """Address of a tensor / array buffer (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    return int(t)


# ---- functions with the names of the C ABI --------------------------------

def lh_default_phys():
    p = lh_phys_desc()
    load().lh_default_phys(ctypes.byref(p))
    return p


def lh_create(mesh, disc, phys, precision, stream=None):
    h = _vp()
    st = load().lh_create(ctypes.byref(mesh), ctypes.byref(disc), ctypes.byref(phys),
                          int(precision), stream, ctypes.byref(h))
    if st != LH_OK:
        raise LaghError(st, "lh_create failed")
    return h


def _check(ctx, st):
    if st != LH_OK:
        raise LaghError(st, load().lh_last_error(ctx).decode())


def lh_destroy(ctx):
    load().lh_destroy(ctx)


def lh_layout(ctx):
    info = lh_layout_info()
    _check(ctx, load().lh_layout(ctx, ctypes.byref(info)))
    return info


def lh_init_state(ctx):
    _check(ctx, load().lh_init_state(ctx))


def lh_set_state(ctx, v, e, x, t=0.0, dt=0.0):
    _check(ctx, load().lh_set_state(ctx, _ptr(v), _ptr(e), _ptr(x), float(t), float(dt)))


def lh_get_state(ctx, v=None, e=None, x=None):
    t = ctypes.c_double()
    dt = ctypes.c_double()
    _check(ctx, load().lh_get_state(ctx, _ptr(v), _ptr(e), _ptr(x), ctypes.byref(t),
                                    ctypes.byref(dt)))
    return t.value, dt.value


def lh_force(ctx, v, e, x, F1, vtest=None, FTv=None, want_dt=True):
    dt = ctypes.c_double()
    _check(ctx, load().lh_force(ctx, _ptr(v), _ptr(e), _ptr(x), _ptr(vtest), _ptr(F1), _ptr(FTv),
                                ctypes.byref(dt) if want_dt else None))
    return dt.value if want_dt else None


def lh_force_sampled(ctx, elem_ids, n, v, e, x, F1_local, vtest=None, FTv_local=None,
                     want_dt=True):
    dt = ctypes.c_double()
    _check(ctx, load().lh_force_sampled(ctx, _ptr(elem_ids), int(n), _ptr(v), _ptr(e), _ptr(x),
                                        _ptr(vtest), _ptr(F1_local), _ptr(FTv_local),
                                        ctypes.byref(dt) if want_dt else None))
    return dt.value if want_dt else None


def lh_mass_apply_v(ctx, a, out):
    _check(ctx, load().lh_mass_apply_v(ctx, _ptr(a), _ptr(out)))


def lh_mass_solve_v(ctx, rhs, out):
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    _check(ctx, load().lh_mass_solve_v(ctx, _ptr(rhs), _ptr(out), ctypes.byref(it),
                                       ctypes.byref(rr)))
    return it.value, rr.value


def lh_precond_apply(ctx, a, out):
    _check(ctx, load().lh_precond_apply(ctx, _ptr(a), _ptr(out)))


def lh_mass_solve_e(ctx, rhs, out):
    _check(ctx, load().lh_mass_solve_e(ctx, _ptr(rhs), _ptr(out)))


def lh_total_energy(ctx):
    E = ctypes.c_double()
    _check(ctx, load().lh_total_energy(ctx, ctypes.byref(E)))
    return E.value


def lh_step_fixed(ctx, dt):
    tau = ctypes.c_double()
    _check(ctx, load().lh_step_fixed(ctx, float(dt), ctypes.byref(tau)))
    return tau.value


def lh_step(ctx, t_final):
    acc = ctypes.c_int32()
    t = ctypes.c_double()
    dt = ctypes.c_double()
    _check(ctx, load().lh_step(ctx, float(t_final), ctypes.byref(acc), ctypes.byref(t),
                               ctypes.byref(dt)))
    return bool(acc.value), t.value, dt.value


def lh_run_to(ctx, t_final, max_steps=2 ** 62, dt_log=None, dt_log_cap=0):
    stats = lh_run_stats()
    st = load().lh_run_to(ctx, float(t_final), int(max_steps), ctypes.byref(stats), _ptr(dt_log),
                          int(dt_log_cap))
    _check(ctx, st)
    return {k: getattr(stats, k) for k, _ in lh_run_stats._fields_}


def lh_force_static(mesh, disc, phys, v, e, x, F1, stream=None, want_dt=True):
    """F.1 of a state with no device allocation (see include/lagh.h); returns
    the time-step estimate.  Raises LaghError on a non-zero status."""
    dt = ctypes.c_double()
    st = load().lh_force_static(ctypes.byref(mesh), ctypes.byref(disc), ctypes.byref(phys),
                                _ptr(v), _ptr(e), _ptr(x), _ptr(F1),
                                ctypes.byref(dt) if want_dt else None, stream)
    if st != LH_OK:
        raise LaghError(st, "lh_force_static failed")
    return dt.value if want_dt else None


# ---- batched form ----------------------------------------------------------

def _bcheck(b, st):
    if st != LH_OK:
        raise LaghError(st, load().lh_batch_last_error(b).decode())


def lh_batch_create(meshes, disc, physs, precision, stream=None, tuning=None):
    """meshes, physs: sequences of lh_mesh_desc / lh_phys_desc (one per
    instance).  tuning: lh_batch_tuning or None."""
    n = len(meshes)
    if len(physs) != n:
        raise ValueError("one physics descriptor per mesh")
    M = (lh_mesh_desc * n)(*meshes)
    Ph = (lh_phys_desc * n)(*physs)
    h = _vp()
    st = load().lh_batch_create(n, M, ctypes.byref(disc), Ph, int(precision), stream,
                                ctypes.byref(tuning) if tuning is not None else None,
                                ctypes.byref(h))
    if st != LH_OK:
        raise LaghError(st, "lh_batch_create failed")
    return h


def lh_batch_destroy(b):
    load().lh_batch_destroy(b)


def lh_batch_last_error(b):
    return load().lh_batch_last_error(b).decode()


def lh_batch_layout(b, n):
    off_v = (ctypes.c_int64 * (n + 1))()
    off_e = (ctypes.c_int64 * (n + 1))()
    info = (lh_layout_info * n)()
    _bcheck(b, load().lh_batch_layout(b, ctypes.addressof(off_v), ctypes.addressof(off_e),
                                      ctypes.addressof(info)))
    return list(off_v), list(off_e), list(info)


def lh_batch_init_state(b):
    _bcheck(b, load().lh_batch_init_state(b))


def lh_batch_set_state(b, v, e, x, t=None, dt=None):
    """t, dt: host float64 arrays (numpy) of n, or None."""
    _bcheck(b, load().lh_batch_set_state(b, _ptr(v), _ptr(e), _ptr(x), _ptr(t), _ptr(dt)))


def lh_batch_get_state(b, v=None, e=None, x=None):
    _bcheck(b, load().lh_batch_get_state(b, _ptr(v), _ptr(e), _ptr(x)))


def lh_batch_query(b, t=None, dt=None, steps=None, rejects=None, cg_iters=None, status=None):
    """Host numpy arrays of n (float64, float64, int64, int64, int64, int32)."""
    _bcheck(b, load().lh_batch_query(b, _ptr(t), _ptr(dt), _ptr(steps), _ptr(rejects),
                                     _ptr(cg_iters), _ptr(status)))


def lh_batch_run_to(b, t_final, max_steps=2 ** 62):
    stats = lh_batch_stats()
    _bcheck(b, load().lh_batch_run_to(b, float(t_final), int(max_steps), ctypes.byref(stats)))
    return {k: getattr(stats, k) for k, _ in lh_batch_stats._fields_}


def lh_batch_step_fixed(b, dt):
    """dt: host float64 numpy array of n."""
    stats = lh_batch_stats()
    _bcheck(b, load().lh_batch_step_fixed(b, _ptr(dt), ctypes.byref(stats)))
    return {k: getattr(stats, k) for k, _ in lh_batch_stats._fields_}


def lh_batch_total_energy(b, out):
    """out: host float64 numpy array of n."""
    _bcheck(b, load().lh_batch_total_energy(b, _ptr(out)))


def lh_batch_force_sampled(b, list_off, elem_ids, F1_local, v=None, e=None, x=None, vtest=None,
                           FTv_local=None, dt_est=None):
    _bcheck(b, load().lh_batch_force_sampled(b, _ptr(list_off), _ptr(elem_ids), _ptr(v), _ptr(e),
                                             _ptr(x), _ptr(vtest), _ptr(F1_local),
                                             _ptr(FTv_local), _ptr(dt_est)))


def lh_batch_autotune(b, reps=2):
    t = lh_batch_tuning()
    _bcheck(b, load().lh_batch_autotune(b, int(reps), ctypes.byref(t)))
    return t


def lh_batch_tuning_get(b):
    t = lh_batch_tuning()
    _bcheck(b, load().lh_batch_tuning_get(b, ctypes.byref(t)))
    return t


def lh_check_conversions(inp, f_out, d_out, split_out=None, stream=None):
    st = load().lh_check_conversions(_ptr(inp), int(inp.numel()), _ptr(f_out), _ptr(d_out),
                                     _ptr(split_out), stream)
    if st != LH_OK:
        raise LaghError(st, "lh_check_conversions failed")


def lh_peak_probe(fp64, iters, sink, stream=None):
    """Launches the FMA-rate probe kernel on stream; returns the flops of the
    launch (the caller times it)."""
    fl = ctypes.c_double()
    st = load().lh_peak_probe(1 if fp64 else 0, int(iters), _ptr(sink), stream, ctypes.byref(fl))
    if st != LH_OK:
        raise LaghError(st, "lh_peak_probe failed")
    return fl.value


def lh_peak_probe_lanes(fp64, lanes, iters, sink, stream=None):
    """The probe with the FMA chains on the first `lanes` lanes of every warp;
    returns the flops of the active lanes (the caller times the launch)."""
    fl = ctypes.c_double()
    st = load().lh_peak_probe_lanes(1 if fp64 else 0, int(lanes), int(iters), _ptr(sink), stream,
                                    ctypes.byref(fl))
    if st != LH_OK:
        raise LaghError(st, "lh_peak_probe_lanes failed")
    return fl.value


def lh_pod(S, m, n, offset, eps, U, sigma, work, stream=None):
    """POD of the column-major m x n snapshot matrix S (device); returns
    (k, sweeps).  Raises LaghError on a non-zero status."""
    k = ctypes.c_int64()
    sw = ctypes.c_int32()
    st = load().lh_pod(_ptr(S), int(m), int(n), _ptr(offset), float(eps), _ptr(U), _ptr(sigma),
                       _ptr(work), ctypes.byref(k), ctypes.byref(sw), stream)
    if st != LH_OK:
        raise LaghError(st, "lh_pod failed")
    return k.value, sw.value


def lh_batch_snapshots(b, ids, cap, Sv, Se, Sx):
    n = len(ids)
    arr = (ctypes.c_int32 * max(n, 1))(*[int(i) for i in ids])
    _bcheck(b, load().lh_batch_snapshots(b, n, arr if n else None, int(cap), _ptr(Sv), _ptr(Se),
                                         _ptr(Sx)))


def lh_batch_snapshot_count(b, n):
    out = (ctypes.c_int64 * n)()
    _bcheck(b, load().lh_batch_snapshot_count(b, out))
    return list(out)


# ---- hyper-reduced online step ----------------------------------------------

def _rcheck(r, st):
    if st != LH_OK:
        raise LaghError(st, load().lh_rom_last_error(r).decode())


def lh_rom_create(ctx, Phi_v, nbv, Phi_e, nbe, Phi_x, nbx, v_os, e_os, x_os, ns_f, ns_g,
                  samples_f=None, samples_g=None):
    import numpy as np
    h = _vp()
    sf = None if samples_f is None else np.ascontiguousarray(samples_f, dtype=np.int64)
    sg = None if samples_g is None else np.ascontiguousarray(samples_g, dtype=np.int64)
    st = load().lh_rom_create(ctx, _ptr(Phi_v), int(nbv), _ptr(Phi_e), int(nbe), _ptr(Phi_x),
                              int(nbx), _ptr(v_os), _ptr(e_os), _ptr(x_os), int(ns_f), int(ns_g),
                              _ptr(sf), _ptr(sg), ctypes.byref(h))
    if st != LH_OK:
        raise LaghError(st, load().lh_last_error(ctx).decode())
    return h


def lh_rom_destroy(r):
    load().lh_rom_destroy(r)


def lh_rom_info(r):
    import numpy as np
    info = lh_rom_info_t()
    _rcheck(r, load().lh_rom_info(r, ctypes.byref(info), None, None, None))
    sf = np.zeros(info.ns_f, dtype=np.int64)
    sg = np.zeros(info.ns_g, dtype=np.int64)
    els = np.zeros(info.n_elems, dtype=np.int32)
    _rcheck(r, load().lh_rom_info(r, None, sf.ctypes.data, sg.ctypes.data, els.ctypes.data))
    return info, sf, sg, els


def lh_rom_set_state(r, vh, eh, xh, t=0.0, dt=0.0):
    _rcheck(r, load().lh_rom_set_state(r, _ptr(vh), _ptr(eh), _ptr(xh), float(t), float(dt)))


def lh_rom_get_state(r, vh, eh, xh):
    t = ctypes.c_double()
    dt = ctypes.c_double()
    _rcheck(r, load().lh_rom_get_state(r, _ptr(vh), _ptr(eh), _ptr(xh), ctypes.byref(t),
                                       ctypes.byref(dt)))
    return t.value, dt.value


def lh_rom_lift(r, v, e, x):
    _rcheck(r, load().lh_rom_lift(r, _ptr(v), _ptr(e), _ptr(x)))


def lh_rom_step_fixed(r, dt):
    tau = ctypes.c_double()
    _rcheck(r, load().lh_rom_step_fixed(r, float(dt), ctypes.byref(tau)))
    return tau.value


def lh_rom_run_to(r, t_final, max_steps=2 ** 62):
    st = lh_run_stats()
    _rcheck(r, load().lh_rom_run_to(r, float(t_final), int(max_steps), ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in lh_run_stats._fields_}
