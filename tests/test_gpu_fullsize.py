"""Parity at the full sizes of the benchmark configurations.

The 64x64 Taylor-Green workload runs through the device-controlled time loop
(one CUDA graph per attempt, the launch mode bench.py times) against the
oracle's own control loop.  The 32^3 point blast and the 256x256 Q3 Gresho
vortex are too large for the oracle to step in seconds, so they are compared
on full force fields and sampled element rows (which the oracle computes
directly), and checked on properties that hold at any size: energy balance,
mirror symmetry of the blast, rotation symmetry of the vortex."""
import numpy as np
import pytest

from paper_2104_11404_gb300 import workloads as W
from tests._pair import dev, gpu_for, host, max_rel, oracle_for, random_state, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_taylor_green_64_graph_run_matches_oracle(precision, tol):
    cfg = W.CONFIGS["tg2d_64"]
    steps = 20
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    stats, log, s = o.run(cfg["t_final"], v, e, x, max_steps=steps)
    assert s == 0 and stats["steps"] == steps
    g = gpu_for(cfg, precision=precision)
    g.init_state()
    dt_log = torch.zeros(100, dtype=torch.float64, device="cuda")
    st = g.run_to(cfg["t_final"], max_steps=steps, dt_log=dt_log)
    assert st["steps"] == steps and st["rejects"] == stats["rejects"]
    assert np.allclose(host(dt_log)[:steps], log, rtol=tol, atol=0)
    vg, eg, xg, t, _ = g.get_state()
    assert abs(t - stats["t"]) <= tol * stats["t"]
    assert rel_l2(v, host(vg)) <= tol and rel_l2(e, host(eg)) <= tol
    assert rel_l2(x, host(xg)) <= tol * 1e-2


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_taylor_green_64_force_field(precision, tol):
    cfg = W.CONFIGS["tg2d_64"]
    o = oracle_for(cfg)
    v, e, x = random_state(o, cfg, seed=64, e_range=(140.0, 160.0))
    w = random_state(o, cfg, seed=65)[0]
    F1o, FTvo, dto, s = o.force(v, e, x, vtest=w)
    assert s == 0
    g = gpu_for(cfg, precision=precision)
    F1, FTv, dt = g.force(dev(v), dev(e), dev(x), vtest=dev(w))
    assert max_rel(F1o, host(F1)) <= tol
    assert max_rel(FTvo, host(FTv)) <= tol
    assert abs(dt - dto) <= max(tol, 1e-6 if precision == "mixed" else 0.0) * dto


def _sample_rows(o, g, cfg, ids, v, e, x, w, tol):
    from tests import _fem_ref as R
    d = cfg["dim"]
    F1l, FTvl, _ = g.force_sampled(dev(ids), dev(v), dev(e), dev(x), vtest=dev(w))
    F1l = host(F1l).reshape(len(ids), d * o.nd1)
    FTvl = host(FTvl).reshape(len(ids), o.nd2)
    mesh = R.CartesianMesh(d, cfg["n"][:d], cfg["order"])
    for s, el in enumerate(ids):
        FK = o.element_force_matrix(int(el), v, e, x)
        cn = mesh.conn(int(el))
        wl = np.concatenate([w[c * o.nnodes + cn] for c in range(d)])
        assert max_rel(FK.sum(axis=1), F1l[s]) <= tol
        assert max_rel(FK.T @ wl, FTvl[s]) <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_sedov3d_32_force_and_sampled_rows(precision, tol):
    cfg = W.CONFIGS["sedov3d_32"]
    o = oracle_for(cfg)
    v, e, x = random_state(o, cfg, seed=32)
    w = random_state(o, cfg, seed=33)[0]
    g = gpu_for(cfg, precision=precision)
    ids = W.element_sample(o.nelem, frac=0.0006, stream=3)  # 20 elements
    _sample_rows(o, g, cfg, ids, v, e, x, w, tol)
    if precision == "fp64":  # the full field once (the oracle takes a few seconds)
        F1o, FTvo, dto, s = o.force(v, e, x, vtest=w)
        F1, FTv, dt = g.force(dev(v), dev(e), dev(x), vtest=dev(w))
        assert max_rel(F1o, host(F1)) <= tol and max_rel(FTvo, host(FTv)) <= tol
        assert abs(dt - dto) <= 1e-12 * dto


@pytest.mark.parametrize("precision,etol,stol", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-4)])
def test_sedov3d_32_steps_conserve_energy_and_mirror_symmetry(precision, etol, stol):
    """From the initial blast: total energy is conserved by RK2-average, and
    the solution stays symmetric under every swap of the axes."""
    cfg = W.CONFIGS["sedov3d_32"]
    g = gpu_for(cfg, precision=precision)
    g.init_state()
    E0 = g.total_energy()
    st = g.run_to(cfg["t_final"], max_steps=5)
    assert st["steps"] == 5
    assert abs(g.total_energy() - E0) <= etol * E0
    v, e, x, _, _ = g.get_state()
    nn = 2 * 32 + 1
    V = host(v).reshape(3, nn, nn, nn)  # [c][z][y][x]
    vmax = np.abs(V).max()
    assert vmax > 0
    # swapping x and y maps v_x(x, y, z) to v_y(y, x, z)
    assert np.abs(V[0] - np.transpose(V[1], (0, 2, 1))).max() <= stol * vmax
    # swapping x and z maps v_x(x, y, z) to v_z(z, y, x)
    assert np.abs(V[0] - np.transpose(V[2], (2, 1, 0))).max() <= stol * vmax


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_gresho_256_q3_force_and_sampled_rows(precision, tol):
    cfg = W.CONFIGS["gresho2d_256"]
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    w = random_state(o, cfg, seed=256)[0]
    g = gpu_for(cfg, precision=precision)
    ids = W.element_sample(o.nelem, frac=0.0003, stream=4)  # 20 elements
    _sample_rows(o, g, cfg, ids, v, e, x, w, tol)
    # The full field on a random state: at the initial vortex F.1 is the small
    # net of pressure terms ~300x larger (exact radial balance), which would
    # measure the conditioning of that cancellation instead of the kernels.
    v, e, x = random_state(o, cfg, seed=257)
    F1o, FTvo, dto, s = o.force(v, e, x, vtest=w)
    F1, FTv, dt = g.force(dev(v), dev(e), dev(x), vtest=dev(w))
    assert max_rel(F1o, host(F1)) <= tol and max_rel(FTvo, host(FTv)) <= tol


@pytest.mark.parametrize("precision,etol,stol", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-4)])
def test_gresho_256_q3_steps_conserve_energy_and_rotation_symmetry(precision, etol, stol):
    """No viscosity: total energy is conserved exactly by RK2-average; the
    vortex on the centred square is invariant under a quarter turn."""
    cfg = W.CONFIGS["gresho2d_256"]
    g = gpu_for(cfg, precision=precision)
    g.init_state()
    E0 = g.total_energy()
    v0, _, _, _, _ = g.get_state()
    st = g.run_to(cfg["t_final"], max_steps=5)
    assert st["steps"] == 5
    assert abs(g.total_energy() - E0) <= etol * E0
    v, e, x, _, _ = g.get_state()
    nn = 3 * 256 + 1
    V = host(v).reshape(2, nn, nn)  # [c][y][x], nodes symmetric about the origin
    vmax = np.abs(V).max()
    # a quarter turn (x, y) -> (-y, x) maps node (i, j) to (n-1-j, i):
    # v_x(R p) = -v_y(p) and v_y(R p) = v_x(p)
    assert np.abs(V[0][:, ::-1].T + V[1]).max() <= stol * vmax
    assert np.abs(V[1][:, ::-1].T - V[0]).max() <= stol * vmax
    # the steady vortex stays close to its initial velocity over 5 steps
    assert rel_l2(host(v0), host(v)) <= 1e-2
