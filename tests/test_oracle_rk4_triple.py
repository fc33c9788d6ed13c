"""Pins of the oracle's RK4 integrator (eq:RK4, eq:RK4coeff, reading R14) and
of its triple-point problem (Section 6.1.4, reading R13).

RK4: the semi-discrete system of eq:fom without viscosity is a smooth ODE, so
a correct RK4 has global error O(dt^4): halving dt divides the error by 16.
A wrong stage weight, a stage evaluated at the wrong state or a stage energy
rate formed with another stage's velocity breaks consistency or order, and the
error ratio drops to 2 or 4.  The same measurement gives 4 for RK2-average,
which shows the test can tell the orders apart.

Triple point: the initial state has closed-form mass and internal energy per
material region; at t = 0 the gas is at rest with equal pressure across the
y = 1.5 interface, so F.1 vanishes at every interior node except those on the
x = 1 interface, where it is the pressure jump times the integral of the node's
hat function over the face.  A z-invariant 3D run equals the 2D run on the
same x-y mesh (the 3D element matrices factor into the 2D ones and the z
direction's, and the z mass matrix reproduces constants).
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as P

import oracle as O
from tests import _fem_ref as R


def _tg(n=6, **kw):
    return O.Oracle(dim=2, nx=n, ny=n, order=2, problem=O.TAYLOR_GREEN, gamma=5.0 / 3.0,
                    visc=0, source=1, **kw)


def _perturbed(o, seed):
    v, e, x = o.init_state()
    rng = np.random.default_rng(seed)
    v = v + 0.05 * rng.normal(size=v.shape)
    v[o.essential_mask()] = 0.0
    e = e * (1.0 + 0.01 * rng.uniform(-1, 1, size=e.shape))
    return v, e, x


def _advance(o, step, T, n, v, e, x):
    v, e, x = v.copy(), e.copy(), x.copy()
    for _ in range(n):
        _, _, st = step(T / n, v, e, x)
        assert st == O.OK
    return np.concatenate([v, e, x])


@pytest.mark.parametrize("which,order", [("rk4", 4), ("rk2avg", 2)])
def test_temporal_order(which, order):
    o = _tg()
    v, e, x = _perturbed(o, seed=3)
    step = o.step_rk4 if which == "rk4" else o.step
    T = 0.004
    ref = _advance(o, step, T, 128, v, e, x)
    errs = [np.linalg.norm(_advance(o, step, T, n, v, e, x) - ref) for n in (4, 8, 16)]
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    want = 2.0 ** order
    for r in ratios:
        assert 0.75 * want < r < 1.25 * want, (which, errs, ratios)


def test_rk4_and_rk2avg_agree_to_their_errors():
    """Both integrate the same ODE: after the same short interval they agree
    to the RK2-average error (O(dt^2)), far below the change of the state."""
    o = _tg()
    v, e, x = _perturbed(o, seed=4)
    T = 0.004
    s0 = np.concatenate([v, e, x])
    a = _advance(o, o.step_rk4, T, 32, v, e, x)
    b = _advance(o, o.step, T, 32, v, e, x)
    assert np.linalg.norm(a - b) < 1e-3 * np.linalg.norm(a - s0)


def test_rk4_run_and_rest_state():
    """lho_run with the RK4 integrator: a uniform gas stays at rest exactly,
    and a blast run obeys the step control (steps taken, energy drift small
    but not at roundoff, unlike RK2-average)."""
    o = O.Oracle(dim=2, nx=4, ny=3, order=2, problem=O.UNIFORM, e_uniform=2.0,
                 integrator=O.RK4)
    v, e, x = o.init_state()
    e0, x0 = e.copy(), x.copy()
    stats, _, st = o.run(0.1, v, e, x)
    assert st == O.OK and stats["steps"] > 0
    assert np.abs(v).max() < 1e-12 and np.abs(e - e0).max() < 1e-12 and np.abs(x - x0).max() < 1e-13
    ob = O.Oracle(dim=2, nx=8, ny=8, order=2, problem=O.SEDOV, integrator=O.RK4)
    v, e, x = ob.init_state()
    stats, log, st = ob.run(0.2, v, e, x)
    assert st == O.OK and stats["t"] == 0.2 and stats["steps"] > 20
    drift = abs(stats["energy"] - stats["energy0"]) / stats["energy0"]
    assert drift < 1e-3


# ---------------------------------------------------------------- triple point

def _triple(dim, n, **kw):
    hi = (7.0, 3.0, 1.5)
    return O.Oracle(dim=dim, nx=n[0], ny=n[1], nz=n[2] if dim == 3 else 1, order=2,
                    problem=O.TRIPLE_POINT, lo=(0.0, 0.0, 0.0), hi=hi, **kw)


@pytest.mark.parametrize("dim,n", [(2, (14, 6)), (3, (7, 6, 2))])
def test_triple_point_initial_mass_and_energy_closed_form(dim, n):
    o = _triple(dim, n)
    v, e, x = o.init_state()
    assert np.all(v == 0.0)
    depth = 1.5 if dim == 3 else 1.0
    # regions: x <= 1 (rho 1, p 1, gamma 1.5); x > 1, y <= 1.5 (rho 1, p 0.1,
    # gamma 1.4); x > 1, y > 1.5 (rho 1/8, p 0.1, gamma 1.5)
    vols = np.array([1.0 * 3.0, 6.0 * 1.5, 6.0 * 1.5]) * depth
    rho = np.array([1.0, 1.0, 0.125])
    p = np.array([1.0, 0.1, 0.1])
    gam = np.array([1.5, 1.4, 1.5])
    mass = float(np.sum(rho * vols))
    internal = float(np.sum(p * vols / (gam - 1.0)))
    ones_e = np.ones(o.ne)
    assert abs(o.mass_apply_e(ones_e).sum() - mass) < 1e-12 * mass
    assert abs(o.mass_apply_v(np.ones(o.nv)).sum() - dim * mass) < 1e-12 * mass
    assert abs(o.total_energy(v, e) - internal) < 1e-12 * internal


def _int01(poly):
    c = P.polyint(poly)
    return P.polyval(1.0, c) - P.polyval(0.0, c)


def test_triple_point_initial_force_is_the_pressure_jump():
    n = (14, 6)
    o = _triple(2, n)
    v, e, x = o.init_state()
    F1, _, dt, st = o.force(v, e, x)
    assert st == O.OK and dt > 0.0
    k = 2
    nn = [m * k + 1 for m in n]
    h = [7.0 / n[0], 3.0 / n[1]]
    w1 = np.array([_int01(c) for c in R.lagrange_polys(R.gauss_lobatto01(k + 1))])

    def hat_int(I, c):
        a = I % k
        val = 0.0
        if I < nn[c] - 1:
            val += w1[a] * h[c]
        if a == 0 and I > 0:
            val += w1[k] * h[c]
        return val

    want = np.zeros(o.nv)
    Ix = int(round(1.0 / h[0])) * k          # node column on x = 1
    for J in range(nn[1]):                    # walls y = 0, 3 leave the x component free
        node = Ix + nn[0] * J
        # -int p div(w e_x) over both sides = -(p_left - p_right) int_face w
        want[node] = -(1.0 - 0.1) * hat_int(J, 1)
    scale = np.abs(want).max()
    assert np.abs(F1 - want).max() < 1e-13 * scale


def test_triple_point_3d_z_invariant_run_equals_2d():
    o2 = _triple(2, (14, 6), visc=0)
    o3 = _triple(3, (14, 6, 2), visc=0)
    v2, e2, x2 = o2.init_state()
    v3, e3, x3 = o3.init_state()
    s2, log2, st2 = o2.run(0.3, v2, e2, x2, max_steps=12)
    s3, log3, st3 = o3.run(0.3, v3, e3, x3, max_steps=12)
    assert st2 == O.OK and st3 == O.OK
    assert np.array_equal(log2 > 0, log3 > 0) and np.allclose(log2, log3, rtol=1e-12, atol=0)
    nn2 = o2.nnodes
    nz = 2 * 2 + 1
    V3 = v3.reshape(3, nz, nn2)
    X3 = x3.reshape(3, nz, nn2)
    scale_v = np.abs(v2).max()
    assert scale_v > 0.01
    assert np.abs(V3[2]).max() < 1e-13 * scale_v           # no motion along z
    for kz in range(nz):
        for c in range(2):
            assert np.abs(V3[c, kz] - v2[c * nn2:(c + 1) * nn2]).max() < 1e-11 * scale_v
            assert np.abs(X3[c, kz] - x2[c * nn2:(c + 1) * nn2]).max() < 1e-12 * 7.0
    # energy: k^3 = 8 dofs per 3D element, constant along z within the element
    E3 = e3.reshape(2, 6, 14, 2, 2, 2)                      # [ez, ey, ex, jz, jy, jx]
    E2 = e2.reshape(6, 14, 2, 2)
    for ez in range(2):
        for jz in range(2):
            assert np.abs(E3[ez, :, :, jz] - E2).max() < 1e-11 * np.abs(E2).max()


def test_triple_point_rk2avg_conserves_energy_with_viscosity():
    o = _triple(2, (14, 6))
    v, e, x = o.init_state()
    E0 = o.total_energy(v, e)
    stats, _, st = o.run(0.5, v, e, x)
    assert st == O.OK and stats["steps"] > 10
    assert abs(stats["energy"] - E0) < 1e-12 * E0
    assert np.abs(v).max() > 0.05
