"""Parity of the CUDA library (through the C ABI) with the CPU oracle.

FP64 path: <= 1e-12 relative per evaluation and per step, <= 1e-8 relative
L2 at final time when the GPU replays the oracle's accepted step sizes.
Mixed path: FP32 stress, so <= 1e-5 relative per force evaluation and
<= 1e-4 relative L2 in velocity and energy at final time, with the total
energy conserved to 1e-10 relative (the FP64 contractions of the FP32
element matrices keep the RK2-average energy balance exact).
"""
import numpy as np
import pytest

from paper_2104_11404_gb300 import workloads as W
from tests._pair import dev, gpu_for, host, max_rel, oracle_for, random_state, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (dim, order, elements) spanning several CTAs and a ragged last CTA
SMALL = [(2, 1, (9, 7, 1)), (2, 2, (5, 7, 1)), (2, 3, (3, 5, 1)), (3, 1, (3, 4, 2)),
         (3, 2, (3, 2, 3))]


def _cfg(dim, k, n, problem=W.SEDOV, visc=1):
    return dict(dim=dim, n=n, order=k, problem=problem, gamma=1.4, lo=(0.0, 0.0, 0.0),
                hi=(1.0, 1.0, 1.0), visc=visc, blast_energy=0.25, t_final=0.1)


@pytest.mark.parametrize("dim,k,n", SMALL)
@pytest.mark.parametrize("visc", [0, 1])
def test_force_fp64(dim, k, n, visc):
    cfg = _cfg(dim, k, n, visc=visc)
    o = oracle_for(cfg)
    g = gpu_for(cfg)
    v, e, x = random_state(o, cfg, seed=100 + dim * 10 + k)
    w = random_state(o, cfg, seed=7)[0]
    F1o, FTvo, dto, st = o.force(v, e, x, vtest=w)
    assert st == 0
    F1, FTv, dt = g.force(dev(v), dev(e), dev(x), vtest=dev(w))
    assert max_rel(F1o, host(F1)) <= 1e-12
    assert max_rel(FTvo, host(FTv)) <= 1e-12
    assert abs(dt - dto) <= 1e-12 * dto


@pytest.mark.parametrize("dim,k,n", SMALL)
def test_force_mixed(dim, k, n):
    cfg = _cfg(dim, k, n)
    o = oracle_for(cfg)
    g = gpu_for(cfg, precision="mixed")
    v, e, x = random_state(o, cfg, seed=200 + dim * 10 + k)
    w = random_state(o, cfg, seed=8)[0]
    F1o, FTvo, dto, _ = o.force(v, e, x, vtest=w)
    F1, FTv, dt = g.force(dev(v), dev(e), dev(x), vtest=dev(w))
    assert max_rel(F1o, host(F1)) <= 1e-5
    assert max_rel(FTvo, host(FTv)) <= 1e-5
    assert abs(dt - dto) <= 1e-5 * dto
    # the energy identity holds to FP64 rounding of the FP32 element matrices
    F1h, FTvh = host(F1), host(FTv)
    assert abs(w @ F1h - FTvh.sum()) <= 1e-13 * np.abs(w).max() * np.abs(F1h).sum()


@pytest.mark.parametrize("dim,k,n", SMALL)
def test_mass_operators(dim, k, n):
    cfg = _cfg(dim, k, n)
    o = oracle_for(cfg)
    g = gpu_for(cfg)
    rng = np.random.default_rng(dim * 100 + k)
    a = rng.normal(size=o.nv)
    assert max_rel(o.mass_apply_v(a), host(g.mass_apply_v(dev(a)))) <= 1e-14
    xo, _, _, st = o.mass_solve_v(a)
    xg, its, rr = g.mass_solve_v(dev(a))
    assert st == 0 and rr <= 1e-14 and its > 0
    assert rel_l2(xo, host(xg)) <= 1e-12
    assert np.all(host(xg)[W.essential_mask(cfg)] == 0.0)
    b = rng.normal(size=o.ne)
    assert max_rel(o.mass_solve_e(b), host(g.mass_solve_e(dev(b)))) <= 1e-13


@pytest.mark.parametrize("dim,k,n", SMALL)
def test_cg_preconditioners_agree(dim, k, n):
    from paper_2104_11404_gb300 import lagh
    cfg = _cfg(dim, k, n)
    o = oracle_for(cfg)
    rng = np.random.default_rng(5 + dim + k)
    b = rng.normal(size=o.nv)
    xo, _, _, _ = o.mass_solve_v(b)
    gt = gpu_for(cfg, phys_overrides={"cg_precond": lagh.LH_PRECOND_TENSOR})
    gj = gpu_for(cfg, phys_overrides={"cg_precond": lagh.LH_PRECOND_JACOBI})
    ge = gpu_for(cfg, phys_overrides={"cg_precond": lagh.LH_PRECOND_EXACT})
    g64 = gpu_for(cfg, phys_overrides={"cg_precond": lagh.LH_PRECOND_TENSOR64})
    xt, it_t, rr_t = gt.mass_solve_v(dev(b))
    xj, it_j, rr_j = gj.mass_solve_v(dev(b))
    xe, it_e, rr_e = ge.mass_solve_v(dev(b))
    x6, it_6, rr_6 = g64.mass_solve_v(dev(b))
    for xg in (xt, xj, xe, x6):
        assert rel_l2(xo, host(xg)) <= 1e-12
    # banded inverse in FP32: a few iterations; in FP64: two; the exact inverse: one
    assert it_e == 1 and rr_e <= 1e-14
    assert it_6 <= 2 and rr_6 <= 1e-14
    assert it_t <= 3 < it_j


@pytest.mark.parametrize("dim,k,n", SMALL)
def test_precond_apply_approximates_mass_inverse(dim, k, n):
    from paper_2104_11404_gb300 import lagh
    cfg = _cfg(dim, k, n)
    o = oracle_for(cfg)
    g = gpu_for(cfg, phys_overrides={"cg_precond": lagh.LH_PRECOND_TENSOR})
    b = np.random.default_rng(11 + dim + k).normal(size=o.nv)
    xo, _, _, _ = o.mass_solve_v(b)
    out = g.zeros_v()
    lagh.lh_precond_apply(g.ctx, dev(b), out)
    z = host(out)
    assert np.all(z[W.essential_mask(cfg)] == 0.0)
    # FP32 banded inverse: close to M_V^{-1} b, not equal
    assert 1e-12 < rel_l2(xo, z) <= 1e-6
    # the exact variant is M_V^{-1} up to rounding
    ge = gpu_for(cfg, phys_overrides={"cg_precond": lagh.LH_PRECOND_EXACT})
    out = ge.zeros_v()
    lagh.lh_precond_apply(ge.ctx, dev(b), out)
    ze = host(out)
    assert np.all(ze[W.essential_mask(cfg)] == 0.0)
    assert rel_l2(xo, ze) <= 1e-13


# 2D meshes whose band passes are narrow (tile kernel): ragged last tiles and
# 17-wide ones (16m + 1 node lines); 64 x 64 Q2 is the Taylor-Green size (128
# CTAs, halos shared across many)
TILED = [(1, (9, 7, 1)), (2, (5, 7, 1)), (3, (3, 5, 1)), (2, (40, 23, 1)), (3, (21, 9, 1)),
         (1, (32, 16, 1)), (2, (64, 64, 1))]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k,n", TILED)
def test_band_tiles_match_line_passes(k, n, precision):
    """The 16 x 16 tile kernel forms the same sums as the x and y line passes,
    in the same order (plain FP32 on the FP64 path, error-free sums with the
    bands' low parts on the mixed path): its preconditioner output is bitwise
    theirs, and a solve and a few steps through either agree to rounding (the
    dot products add their block partials over a different tiling)."""
    from paper_2104_11404_gb300 import lagh
    cfg = _cfg(2, k, n)
    o = oracle_for(cfg)
    over = {"cg_cluster": -1}
    gt = gpu_for(cfg, precision, phys_overrides=dict(over))
    gl = gpu_for(cfg, precision, phys_overrides=dict(over, cg_tiles=-1))
    b = np.random.default_rng(40 + k).normal(size=o.nv)
    zt, zl = gt.zeros_v(), gl.zeros_v()
    lagh.lh_precond_apply(gt.ctx, dev(b), zt)
    lagh.lh_precond_apply(gl.ctx, dev(b), zl)
    assert torch.equal(zt, zl) and float(zt.abs().max()) > 0
    xt, it_t, rr_t = gt.mass_solve_v(dev(b))
    xl, it_l, rr_l = gl.mass_solve_v(dev(b))
    xo, _, _, _ = o.mass_solve_v(b)
    assert abs(it_t - it_l) <= 1 and rr_t <= 1e-14
    if precision == "mixed":  # error-free band sums: two iterations reach 1e-14
        assert it_t <= 2 and it_l <= 2, (it_t, it_l)
    assert rel_l2(xo, host(xt)) <= 1e-12 and rel_l2(host(xl), host(xt)) <= 1e-13
    its = []
    for g in (gt, gl):
        g.init_state()
        st = g.run_to(cfg["t_final"], max_steps=4)
        assert st["steps"] == 4
        its.append(st["cg_iters"])
    # the same iterations (a tile reading a neighbour's new residual as its
    # halo would still converge, in more iterations)
    assert abs(its[0] - its[1]) <= 2, its
    vt, et, _, tt, _ = gt.get_state()
    vl, el, _, tl, _ = gl.get_state()
    assert abs(tt - tl) <= 1e-13 * tl
    tol = 1e-11 if precision == "fp64" else 1e-9
    assert rel_l2(host(vl), host(vt)) <= tol and rel_l2(host(el), host(et)) <= tol


def _per_step(cfg, nsteps, precision="fp64", tol=1e-12):
    """Each step from the same state: the oracle advances its own trajectory
    under step control; the GPU is set to the oracle's state, takes the same
    step and is compared field by field (eq:relerrors)."""
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    g = gpu_for(cfg, precision=precision)
    g.init_state()
    vg, eg, xg, t, _ = g.get_state()
    assert max_rel(v, host(vg)) <= 1e-15 and max_rel(e, host(eg)) <= 1e-15
    assert max_rel(x, host(xg)) <= 1e-15
    worst = 0.0
    dt_next = 0.0
    for _ in range(nsteps):
        g.set_state(v, e, x, t=0.0, dt=1.0)
        stats, log, st = o.run(1.0, v, e, x, dt=dt_next, max_steps=1)
        assert st == 0
        dt_next = stats["dt"]
        tau_g = g.step_fixed(float(log[0]))
        vg, eg, xg, _, _ = g.get_state()
        for a, b in ((v, vg), (e, eg), (x, xg)):
            worst = max(worst, rel_l2(a, host(b)))
    assert worst <= tol, worst


@pytest.mark.parametrize("name,n,steps", [("sedov2d_8", (8, 8), 12), ("tg2d_64", (16, 16), 8),
                                           ("gresho2d_256", (8, 8), 6),
                                           ("sedov3d_32", (4, 4, 4), 6)])
def test_steps_fp64_per_step(name, n, steps):
    cfg = W.scaled(name, n=n)
    _per_step(cfg, steps)


@pytest.mark.parametrize("name,n,steps", [("sedov2d_8", (8, 8), 6), ("tg2d_64", (16, 16), 6),
                                           ("gresho2d_256", (8, 8), 4)])
def test_steps_mixed_per_step(name, n, steps):
    cfg = W.scaled(name, n=n)
    _per_step(cfg, steps, precision="mixed", tol=1e-5)


def test_sedov_full_run_replay_fp64():
    """2D blast to t = 0.8: the GPU replays the oracle's accepted step sizes;
    final fields within 1e-8 (eq:relerrors) and energy conserved."""
    cfg = W.CONFIGS["sedov2d_8"]
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    stats, log, st = o.run(cfg["t_final"], v, e, x)
    assert st == 0
    g = gpu_for(cfg)
    g.init_state()
    E0 = g.total_energy()
    for dt in log:
        g.step_fixed(float(dt))
    vg, eg, xg, t, _ = g.get_state()
    assert abs(t - cfg["t_final"]) < 1e-12
    assert rel_l2(v, host(vg)) <= 1e-8
    assert rel_l2(e, host(eg)) <= 1e-8
    assert rel_l2(x, host(xg)) <= 1e-8
    assert abs(g.total_energy() - E0) <= 1e-12 * E0


def test_sedov_free_running_control_fp64():
    """Device-side step control against the oracle's control loop."""
    cfg = W.CONFIGS["sedov2d_8"]
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    stats, log, st = o.run(cfg["t_final"], v, e, x)
    g = gpu_for(cfg)
    g.init_state()
    dt_log = torch.zeros(10000, dtype=torch.float64, device="cuda")
    gs = g.run_to(cfg["t_final"], dt_log=dt_log)
    assert gs["t"] == cfg["t_final"]
    assert gs["steps"] == stats["steps"] and gs["rejects"] == stats["rejects"]
    assert np.allclose(host(dt_log)[: gs["steps"]], log, rtol=1e-10, atol=0)
    vg, eg, xg, _, _ = g.get_state()
    assert rel_l2(v, host(vg)) <= 1e-8 and rel_l2(e, host(eg)) <= 1e-8
    assert abs(gs["energy"] - gs["energy0"]) <= 1e-12 * gs["energy0"]


def test_taylor_green_mixed_accuracy_and_energy():
    cfg = W.scaled("tg2d_64", n=(16, 16), t_final=0.05)
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    stats, log, st = o.run(cfg["t_final"], v, e, x)
    g = gpu_for(cfg, precision="mixed")
    g.init_state()
    for dt in log:
        g.step_fixed(float(dt))
    vg, eg, xg, _, _ = g.get_state()
    assert rel_l2(v, host(vg)) <= 1e-4
    assert rel_l2(e, host(eg)) <= 1e-4
    assert rel_l2(x, host(xg)) <= 1e-6


def test_sedov_mixed_energy_drift():
    cfg = W.CONFIGS["sedov2d_8"]
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    stats, log, st = o.run(0.3, v, e, x)
    g = gpu_for(cfg, precision="mixed")
    g.init_state()
    E0 = g.total_energy()
    for dt in log:
        g.step_fixed(float(dt))
    assert abs(g.total_energy() - E0) <= 1e-10 * E0
    vg, eg, xg, _, _ = g.get_state()
    assert rel_l2(v, host(vg)) <= 1e-4 and rel_l2(e, host(eg)) <= 1e-4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("dim,k,n", [(2, 2, (6, 5, 1)), (3, 2, (3, 3, 2)), (2, 3, (4, 3, 1))])
def test_force_sampled(dim, k, n, precision, tol):
    cfg = _cfg(dim, k, n)
    o = oracle_for(cfg)
    g = gpu_for(cfg, precision=precision)
    v, e, x = random_state(o, cfg, seed=31)
    w = random_state(o, cfg, seed=32)[0]
    ids = W.element_sample(o.nelem, frac=0.3, stream=dim * 10 + k)
    F1l, FTvl, dt = g.force_sampled(dev(ids), dev(v), dev(e), dev(x), vtest=dev(w))
    F1l = host(F1l).reshape(len(ids), dim * o.nd1)
    FTvl = host(FTvl).reshape(len(ids), o.nd2)
    from tests import _fem_ref as R
    mesh = R.CartesianMesh(dim, n[:dim], k)
    taus = []
    for s, el in enumerate(ids):
        FK = o.element_force_matrix(int(el), v, e, x)
        cn = mesh.conn(int(el))
        wl = np.concatenate([w[c * o.nnodes + cn] for c in range(dim)])
        assert max_rel(FK.sum(axis=1), F1l[s]) <= tol
        assert max_rel(FK.T @ wl, FTvl[s]) <= tol
    # empty list: nothing to do
    F1e, _, _ = g.force_sampled(dev(np.zeros(0, dtype=np.int32)), dev(v), dev(e), dev(x))
    assert F1e.numel() == 0


def test_device_errors_are_reported():
    from paper_2104_11404_gb300 import lagh
    cfg = _cfg(2, 2, (4, 4, 1))
    o = oracle_for(cfg)
    g = gpu_for(cfg)
    v, e, x = o.init_state()
    # inverted element: swap two corner nodes of element 0
    xt = x.copy()
    nn = 9
    xt[0], xt[2] = xt[2], xt[0]
    with pytest.raises(lagh.LaghError) as ei:
        g.force(dev(v), dev(e), dev(xt))
    assert ei.value.status == lagh.LH_ETANGLED
    en = e.copy()
    en[5] = np.nan
    with pytest.raises(lagh.LaghError) as ei:
        g.force(dev(v), dev(en), dev(x))
    assert ei.value.status == lagh.LH_ENONFINITE
    g1 = gpu_for(cfg, cg_maxit=1, phys_overrides={"cg_precond": lagh.LH_PRECOND_JACOBI})
    with pytest.raises(lagh.LaghError) as ei:
        g1.mass_solve_v(dev(np.random.default_rng(0).normal(size=o.nv)))
    assert ei.value.status == lagh.LH_ECG
    g2 = gpu_for(cfg, phys_overrides={"dt_min_frac": 0.05})
    g2.init_state()
    g2.set_state(dev(v), dev(e), dev(x), t=0.0, dt=0.5)
    with pytest.raises(lagh.LaghError) as ei:
        g2.run_to(1.0)
    assert ei.value.status == lagh.LH_EDTMIN


def test_invalid_descriptors():
    from paper_2104_11404_gb300 import lagh
    cfg = _cfg(3, 3, (2, 2, 2))
    with pytest.raises(lagh.LaghError) as ei:
        gpu_for(cfg)
    assert ei.value.status == lagh.LH_EUNSUPPORTED
    cfg = _cfg(2, 2, (0, 2, 1))
    with pytest.raises(lagh.LaghError) as ei:
        gpu_for(cfg)
    assert ei.value.status == lagh.LH_EINVAL


def test_integer_pipe_conversions_match_ieee_casts():
    """The FP32 paths convert with integer operations; they must equal the
    IEEE 754 casts bit for bit (nearest-even rounding to FP32, subnormal
    results included, and exact widening back to FP64)."""
    from paper_2104_11404_gb300 import lagh
    rng = np.random.default_rng(2)
    vals = [0.0, -0.0, 1.0, -1.0, 0.1, 1.0 / 3.0, np.pi, 1e-30, -1e30, 3.4028234663852886e38,
            3.4028235677973366e38, 1e39, -1e39, np.inf, -np.inf, 1.1754943508222875e-38,
            1e-40, 5e-324, 2.2250738585072014e-308]
    # ties and the carry into the exponent: 1 + (2k+1) 2^-24 and (2 - 2^-24)
    vals += [1.0 + (2 * k + 1) * 2.0 ** -24 for k in range(8)]
    vals += [2.0 - 2.0 ** -24, 2.0 - 2.0 ** -25, 1.0 + 2.0 ** -24 + 2.0 ** -60]
    vals += list(rng.normal(size=2000) * 10.0 ** rng.integers(-30, 30, size=2000))
    vals += list(rng.uniform(-1, 1, size=2000))
    # the FP32 subnormal range: its grid 2^-149, ties, the carry into 2^-126
    tiny = 2.0 ** -149
    vals += [tiny, -tiny, 0.5 * tiny, 1.5 * tiny, 2.5 * tiny, 0.5000001 * tiny, 0.4999999 * tiny,
             (2.0 ** 23 - 0.5) * tiny, (2.0 ** 23 - 0.25) * tiny, 1e-45, 7e-46, -1e-41]
    vals += list(rng.uniform(-1, 1, size=2000) * 10.0 ** rng.integers(-46, -37, size=2000))
    a = np.array(vals, dtype=np.float64)
    f = torch.empty(len(a), dtype=torch.float32, device="cuda")
    d = torch.empty(len(a), dtype=torch.float64, device="cuda")
    sp = torch.empty(len(a), dtype=torch.float64, device="cuda")
    lagh.lh_check_conversions(dev(a), f, d, sp)
    torch.cuda.synchronize()
    fh, dh, sph = host(f), host(d), host(sp)
    with np.errstate(over="ignore"):
        ref = a.astype(np.float32)
    assert np.array_equal(fh.view(np.uint32), ref.view(np.uint32))
    assert np.any((fh != 0) & (np.abs(fh) < np.finfo(np.float32).tiny))  # subnormals reached
    # widening is exact
    assert np.array_equal(dh.view(np.uint64), fh.astype(np.float64).view(np.uint64))
    # the two-float split holds 48 bits where the value is in the FP32 range
    mid = np.isfinite(a) & (np.abs(a) > 1e-22) & (np.abs(a) < 1e38)
    assert np.all(np.abs(sph[mid] - a[mid]) <= 2.0 ** -47 * np.abs(a[mid]))
    nan = torch.tensor([np.nan], dtype=torch.float64, device="cuda")
    f1 = torch.empty(1, dtype=torch.float32, device="cuda")
    d1 = torch.empty(1, dtype=torch.float64, device="cuda")
    lagh.lh_check_conversions(nan, f1, d1)
    assert np.isnan(host(f1)[0]) and np.isnan(host(d1)[0])


@pytest.mark.parametrize("name,n", [("tg2d_64", (24, 20)), ("sedov2d_8", (8, 8)),
                                    ("gresho2d_256", (10, 12))])
def test_cluster_cg_matches_kernel_chain(name, n):
    """The velocity solve of a small 2D problem as one cluster launch gives
    the solution of the kernel chain (same algorithm, sums in another order),
    with the same iteration counts, through single solves and a graph run."""
    cfg = W.scaled(name, n=n)
    o = oracle_for(cfg)
    rng = np.random.default_rng(17)
    b = rng.normal(size=o.nv)
    xo, _, _, _ = o.mass_solve_v(b)
    gc = gpu_for(cfg, phys_overrides={"cg_cluster": 1})       # cluster form (forced)
    gk = gpu_for(cfg, phys_overrides={"cg_cluster": -1})
    xc, itc, rrc = gc.mass_solve_v(dev(b))
    xk, itk, rrk = gk.mass_solve_v(dev(b))
    assert abs(itc - itk) <= 1 and rrc <= 1e-14 and rrk <= 1e-14
    assert rel_l2(xo, host(xc)) <= 1e-12 and rel_l2(host(xk), host(xc)) <= 1e-13
    gc.init_state()
    gk.init_state()
    sc = gc.run_to(cfg["t_final"], max_steps=6)
    sk = gk.run_to(cfg["t_final"], max_steps=6)
    # a solve that converges right at the tolerance may take one more iteration
    # in either form (the sums differ in rounding order)
    assert sc["steps"] == sk["steps"]
    assert abs(sc["cg_iters"] - sk["cg_iters"]) <= 2 * (sc["steps"] + sc["rejects"])
    vc, ec, _, _, _ = gc.get_state()
    vk, ek, _, _, _ = gk.get_state()
    assert rel_l2(host(vk), host(vc)) <= 1e-10 and rel_l2(host(ek), host(ec)) <= 1e-10


def test_lane_probe_counts_active_lanes_only():
    """The FMA probe on a part of every warp reports the flops of the active
    lanes: 2 x 8 chains x iterations x 8 blocks per SM x 8 warps x lanes."""
    from paper_2104_11404_gb300 import lagh
    sink = torch.zeros(8 * 1024, dtype=torch.float64, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for lanes in (32, 4, 1):
        fl = lagh.lh_peak_probe_lanes(True, lanes, 10, sink, torch.cuda.current_stream().cuda_stream)
        assert fl == 2.0 * 8 * 10 * 8 * sms * 8 * lanes
    torch.cuda.synchronize()
    assert float(sink.abs().sum()) == 0.0
