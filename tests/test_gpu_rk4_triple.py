"""RK4 integrator (eq:RK4, eq:RK4coeff) and the triple-point problem
(Section 6.1.4) on the GPU against the oracle.

RK4: one step from seeded random states with given step sizes, element by
element against the oracle's RK4 step (FP64 1e-12, mixed 1e-5), and a run
under the step control of Section 2.2.3 (the same accepted steps, final
fields to 1e-10).  Triple point: per-element density, pressure and adiabatic
index; force (F.1, F^T v, estimate) on the initial and on a perturbed state,
replayed steps, a free-running run against the oracle's (FP64 1e-8 relative
L2 at the final time, the same steps), the mixed path within 1e-4, total
energy conserved by RK2-average."""
import numpy as np
import pytest

from paper_2104_11404_gb300 import workloads as W
from tests._pair import dev, gpu_for, host, max_rel, oracle_for, random_state, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sedov(dim, n, k=2, **over):
    c = dict(dim=dim, n=tuple(n) + (1,) * (3 - len(n)), order=k, problem=W.SEDOV, gamma=1.4,
             lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1, blast_energy=0.25)
    c.update(over)
    return c


RK4_CASES = [
    ("sedov2d_q2", _sedov(2, (6, 5), integrator=W.RK4)),
    ("sedov2d_q1", _sedov(2, (5, 4), k=1, integrator=W.RK4)),
    ("tg2d_q2_source", dict(W.scaled("tg2d_64", n=(5, 4)), integrator=W.RK4)),
    ("gresho2d_q3", dict(W.scaled("gresho2d_256", n=(4, 4)), integrator=W.RK4)),
    ("sedov3d_q2", _sedov(3, (3, 3, 2), integrator=W.RK4)),
]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("name,cfg", RK4_CASES, ids=[c[0] for c in RK4_CASES])
def test_rk4_step_matches_oracle(name, cfg, precision, tol):
    o = oracle_for(cfg)
    v, e, x = random_state(o, cfg, seed=91)
    # wall nodes stay on their walls (as in every state the integrator makes):
    # the mixed path's reference pressure relies on the box boundary
    x0 = o.init_state()[2]
    ess = W.essential_mask(cfg)
    x[ess] = x0[ess]
    g = gpu_for(cfg, precision)
    g.set_state(dev(v), dev(e), dev(x))
    for dt in (1.1e-3, 0.7e-3):
        tau_o, _, st = o.step_rk4(dt, v, e, x)
        assert st == 0
        tau_g = g.step_fixed(dt)
        assert abs(tau_g - tau_o) <= max(tol, 1e-12) * tau_o
        vg, eg, xg, _, _ = g.get_state()
        assert max_rel(v, host(vg)) <= tol
        assert max_rel(e, host(eg)) <= tol
        assert max_rel(x, host(xg)) <= tol * 1e-2
    g.close()


def test_rk4_free_running_matches_oracle():
    cfg = _sedov(2, (8, 8), integrator=W.RK4)
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    st_o, log_o, s = o.run(0.2, v, e, x)
    assert s == 0
    g = gpu_for(cfg, "fp64")
    g.init_state()
    st = g.run_to(0.2)
    assert st["steps"] == st_o["steps"] and st["rejects"] == st_o["rejects"]
    vg, eg, xg, t, _ = g.get_state()
    assert t == 0.2
    for a, b in ((v, vg), (e, eg), (x, xg)):
        assert rel_l2(a, host(b)) <= 1e-10
    g.close()


def _triple(dim, n, **over):
    base = W.CONFIGS["triple3d_28"]
    c = dict(base, dim=dim, n=tuple(n) + (1,) * (3 - len(n)))
    c.update(over)
    return c


TRIPLE_CASES = [("2d_14x6", _triple(2, (14, 6))), ("3d_7x6x2", _triple(3, (7, 6, 2)))]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("name,cfg", TRIPLE_CASES, ids=[c[0] for c in TRIPLE_CASES])
def test_triple_point_force_matches_oracle(name, cfg, precision, tol):
    o = oracle_for(cfg)
    g = gpu_for(cfg, precision)
    v0, e0, x0 = o.init_state()
    g.init_state()
    vg, eg, xg, _, _ = g.get_state()
    assert np.array_equal(host(xg), x0) and np.array_equal(host(vg), v0)
    assert max_rel(e0, host(eg)) <= 1e-15
    for v, e, x in ((v0, e0, x0), random_state(o, cfg, seed=17, e_range=(0.5, 4.0))):
        rng = np.random.default_rng(3)
        vt = rng.normal(size=o.nv)
        F1o, FTvo, dto, st = o.force(v, e, x, vtest=vt)
        assert st == 0
        F1, FTv, dtg = g.force(dev(v), dev(e), dev(x), vtest=dev(vt))
        assert max_rel(F1o, host(F1)) <= tol
        assert max_rel(FTvo, host(FTv)) <= tol
        assert abs(dtg - dto) <= max(tol, 1e-13) * dto
    g.close()


@pytest.mark.parametrize("name,cfg", TRIPLE_CASES, ids=[c[0] for c in TRIPLE_CASES])
def test_triple_point_run_matches_oracle(name, cfg):
    t_final = 0.5 if cfg["dim"] == 2 else 0.3
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    E0 = o.total_energy(v, e)
    st_o, log_o, s = o.run(t_final, v, e, x)
    assert s == 0 and st_o["steps"] > 10
    g = gpu_for(cfg, "fp64")
    g.init_state()
    for dt in log_o:  # replay of the oracle's step sizes
        g.step_fixed(float(dt))
    vg, eg, xg, _, _ = g.get_state()
    for a, b in ((v, vg), (e, eg), (x, xg)):
        assert rel_l2(a, host(b)) <= 1e-8
    g.init_state()  # free running: the same decisions
    st = g.run_to(t_final)
    assert st["steps"] == st_o["steps"] and st["rejects"] == st_o["rejects"]
    vg, eg, xg, _, _ = g.get_state()
    for a, b in ((v, vg), (e, eg), (x, xg)):
        assert rel_l2(a, host(b)) <= 1e-8
    assert abs(g.total_energy() - E0) <= 1e-12 * E0
    g.close()
    gm = gpu_for(cfg, "mixed")
    gm.init_state()
    gm.run_to(t_final)
    vm, em, xm, tm, _ = gm.get_state()
    assert tm == t_final
    assert rel_l2(v, host(vm)) <= 1e-4 and rel_l2(e, host(em)) <= 1e-4
    assert abs(gm.total_energy() - E0) <= 1e-10 * E0
    gm.close()


def test_batch_rejects_triple_point_and_rk4():
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300.batch import Batch
    for cfg in (_triple(2, (14, 6)), _sedov(2, (6, 6), integrator=W.RK4)):
        with pytest.raises(lagh.LaghError) as ei:
            Batch([cfg], precision="fp64")
        assert ei.value.status == lagh.LH_EUNSUPPORTED
