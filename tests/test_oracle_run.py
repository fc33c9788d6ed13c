"""Integrated pins of the oracle's time stepping (eq:RK2-avg, Section 2.2.3):
exact discrete energy conservation of RK2-average, rest states, mirror
symmetry of the blast, manufactured and steady exact solutions, and the step
control bookkeeping."""
import numpy as np
import pytest

import oracle as O


def _sedov(n=8, **kw):
    return O.Oracle(dim=2, nx=n, ny=n, order=2, problem=O.SEDOV, **kw)


def test_sedov_total_energy_conserved_over_full_run():
    o = _sedov()
    v, e, x = o.init_state()
    E0 = o.total_energy(v, e)
    assert abs(E0 - 0.25) < 1e-15
    stats, log, st = o.run(0.8, v, e, x)
    assert st == O.OK and stats["t"] == 0.8
    assert abs(stats["energy"] - E0) <= 1e-12 * E0
    # the loop is not trivially short: steps were taken and some were redone
    assert stats["steps"] > 100 and stats["rejects"] >= 1
    assert abs(log.sum() - 0.8) < 1e-12


def test_midpoint_energy_fails_where_rk2_average_conserves():
    """A plausible mistake (midpoint RK2 energy update with F^T v^n) is not
    conservative; the test checks the conservation test can see it."""
    o = _sedov()
    v, e, x = o.init_state()
    o.run(0.05, v, e, x)
    dt = 2e-3
    E0 = o.total_energy(v, e)
    v1, e1, x1 = v.copy(), e.copy(), x.copy()
    o.step(dt, v1, e1, x1)
    assert abs(o.total_energy(v1, e1) - E0) < 1e-14 * E0
    # midpoint update rebuilt from the oracle's own force and mass solves
    F1, FTv, _, _ = o.force(v, e, x, vtest=v)
    a = o.mass_solve_v(-F1)[0]
    vh = v + 0.5 * dt * a
    eh = e + 0.5 * dt * o.mass_solve_e(FTv)
    xh = x + 0.5 * dt * vh
    F1h, FTvh, _, _ = o.force(vh, eh, xh, vtest=vh)
    v2 = v + dt * o.mass_solve_v(-F1h)[0]
    e2 = e + dt * o.mass_solve_e(FTvh)
    assert abs(o.total_energy(v2, e2) - E0) > 1e-9 * E0


def test_sedov_mirror_symmetry():
    n = 8
    o = _sedov(n)
    v, e, x = o.init_state()
    stats, _, st = o.run(0.3, v, e, x)
    assert st == O.OK
    nn = 2 * n + 1
    vx, vy = v[:nn * nn].reshape(nn, nn), v[nn * nn:].reshape(nn, nn)
    xx, xy = x[:nn * nn].reshape(nn, nn), x[nn * nn:].reshape(nn, nn)
    scale = np.abs(v).max()
    assert scale > 0.1
    assert np.abs(vx - vy.T).max() <= 1e-12 * scale
    assert np.abs(xx - xy.T).max() <= 1e-12
    # e: element (i,j) <-> (j,i), local dofs transposed
    E = e.reshape(n, n, 2, 2)  # [ey, ex, jy, jx]
    assert np.abs(E - E.transpose(1, 0, 3, 2)).max() <= 1e-12 * np.abs(e).max()


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 1), (2, 3)])
def test_uniform_gas_stays_at_rest(dim, k):
    o = O.Oracle(dim=dim, nx=4, ny=3, nz=2, order=k, problem=O.UNIFORM, e_uniform=2.0)
    v, e, x = o.init_state()
    x0, e0 = x.copy(), e.copy()
    for _ in range(5):
        tau, _, st = o.step(1e-2, v, e, x)
        assert st == O.OK
    # rounding noise only (no viscosity acts on it: reading R3's compression
    # floor), growing no further than a few ulps of the sound-speed scale
    assert np.abs(v).max() < 5e-14
    assert np.abs(x - x0).max() < 1e-15
    assert np.abs(e - e0).max() < 1e-13


def _tg_error(n, t_final=0.1, source=1):
    o = O.Oracle(dim=2, nx=n, ny=n, order=2, problem=O.TAYLOR_GREEN, gamma=5.0 / 3.0, visc=0,
                 source=source)
    v, e, x = o.init_state()
    stats, _, st = o.run(t_final, v, e, x)
    assert st == O.OK
    nn = 2 * n + 1
    X, Y = x[:nn * nn], x[nn * nn:]
    vex = np.sin(np.pi * X) * np.cos(np.pi * Y)
    vey = -np.cos(np.pi * X) * np.sin(np.pi * Y)
    err = np.sqrt(np.sum((v[:nn * nn] - vex) ** 2 + (v[nn * nn:] - vey) ** 2)
                  / np.sum(vex ** 2 + vey ** 2))
    return err, o, v, e, x


def test_taylor_green_manufactured_solution_converges():
    e4, *_ = _tg_error(4)
    e8, *_ = _tg_error(8)
    e16, *_ = _tg_error(16)
    assert e8 < 0.3 * e4 and e16 < 0.3 * e8      # at least second order
    assert e16 < 1e-2


def test_taylor_green_source_matters():
    with_src, o, _, e, x = _tg_error(8, t_final=0.2)
    without, *_ = _tg_error(8, t_final=0.2, source=0)
    assert with_src < without


def test_taylor_green_source_formula():
    """int rho e_src phi_j against a fine independent quadrature of
    e_src = v.grad(e) of the exact solution (rho = 1, gamma = 5/3)."""
    o = O.Oracle(dim=2, nx=2, ny=2, order=2, problem=O.TAYLOR_GREEN, gamma=5.0 / 3.0)
    v, e, x = o.init_state()
    src = o.energy_source(x)
    from tests import _fem_ref as R
    qp, qw = R.gauss_legendre01(12)
    L, _ = R.tensor_basis(R.gauss_legendre01(2)[0], qp, 2)
    W = R.tensor_weights(qw, 2)
    Q = np.array([[qp[q % 12], qp[q // 12]] for q in range(144)])
    want = []
    for el in range(4):
        ex, ey = el % 2, el // 2
        X, Y = 0.5 * (ex + Q[:, 0]), 0.5 * (ey + Q[:, 1])
        vx = np.sin(np.pi * X) * np.cos(np.pi * Y)
        vy = -np.cos(np.pi * X) * np.sin(np.pi * Y)
        dpx = -0.5 * np.pi * np.sin(2 * np.pi * X)
        dpy = -0.5 * np.pi * np.sin(2 * np.pi * Y)
        esrc = (vx * dpx + vy * dpy) / (2.0 / 3.0)
        want.append(0.25 * (W * esrc) @ L)
    want = np.concatenate(want)
    # the oracle integrates with 4x4 points: quadrature error only
    assert np.allclose(src, want, atol=2e-3 * np.abs(want).max())
    assert np.abs(src).max() > 0.05


def _gresho_p(r):
    r = np.asarray(r, dtype=float)
    return np.where(r < 0.2, 5 + 12.5 * r ** 2,
                    np.where(r < 0.4, 9 - 4 * np.log(0.2) + 12.5 * r ** 2 - 20 * r + 4 * np.log(r),
                             3 + 4 * np.log(2.0)))


def test_gresho_pressure_reading_is_continuous_and_balanced():
    assert abs(_gresho_p(0.2 - 1e-12) - _gresho_p(0.2)) < 1e-9
    assert abs(_gresho_p(0.4 - 1e-12) - _gresho_p(0.4)) < 1e-9
    assert abs(_gresho_p(0.2) - 5.5) < 1e-12
    # radial balance dp/dr = v_phi^2 / r
    for r in (0.05, 0.15, 0.25, 0.35, 0.45):
        vphi = 5 * r if r < 0.2 else (2 - 5 * r if r < 0.4 else 0.0)
        dp = (_gresho_p(r + 1e-6) - _gresho_p(r - 1e-6)) / 2e-6
        assert abs(dp - vphi ** 2 / r) < 1e-6
    o = O.Oracle(dim=2, nx=4, ny=4, order=3, problem=O.GRESHO, gamma=5.0 / 3.0, visc=0,
                 lo=[-0.5, -0.5, 0], hi=[0.5, 0.5, 1])
    v, e, x = o.init_state()
    # e at the L2 nodes equals p / ((gamma - 1) rho)
    from tests import _fem_ref as R
    g = R.gauss_legendre01(3)[0]
    for el in range(16):
        ex, ey = el % 4, el // 4
        for j in range(9):
            X = -0.5 + 0.25 * (ex + g[j % 3])
            Y = -0.5 + 0.25 * (ey + g[j // 3])
            assert abs(e[el * 9 + j] - _gresho_p(np.hypot(X, Y)) / (2.0 / 3.0)) < 1e-12


def _gresho_error(n, t_final=0.05):
    o = O.Oracle(dim=2, nx=n, ny=n, order=3, problem=O.GRESHO, gamma=5.0 / 3.0, visc=0,
                 lo=[-0.5, -0.5, 0], hi=[0.5, 0.5, 1])
    v, e, x = o.init_state()
    E0 = o.total_energy(v, e)
    stats, _, st = o.run(t_final, v, e, x)
    assert st == O.OK
    nn = 3 * n + 1
    X, Y = x[:nn * nn], x[nn * nn:]
    r = np.hypot(X, Y)
    vp = np.where(r < 0.2, 5 * r, np.where(r < 0.4, 2 - 5 * r, 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        vex = np.where(r > 0, -vp * Y / r, 0.0)
        vey = np.where(r > 0, vp * X / r, 0.0)
    err = np.sqrt(np.sum((v[:nn * nn] - vex) ** 2 + (v[nn * nn:] - vey) ** 2)
                  / np.sum(vex ** 2 + vey ** 2))
    return err, abs(stats["energy"] - E0) / E0


def test_gresho_steady_vortex_converges_and_conserves():
    e8, d8 = _gresho_error(8)
    e16, d16 = _gresho_error(16)
    assert e16 < 0.5 * e8 and e16 < 2e-2
    assert d8 < 1e-12 and d16 < 1e-12


def test_replaying_accepted_steps_reproduces_the_run():
    o = _sedov(6)
    v, e, x = o.init_state()
    v1, e1, x1 = v.copy(), e.copy(), x.copy()
    stats, log, st = o.run(0.2, v1, e1, x1)
    assert st == O.OK
    for dt in log:
        tau, _, st = o.step(dt, v, e, x)
        assert st == O.OK and dt < tau
    assert np.array_equal(v, v1) and np.array_equal(e, e1) and np.array_equal(x, x1)


def test_step_control_rules():
    """Section 2.2.3: a step with dt >= tau is redone with beta1 dt; a step
    with dt <= gamma tau lets the next one grow by beta2."""
    o = _sedov(6)
    v, e, x = o.init_state()
    _, _, tau0, _ = o.force(v, e, x)
    # reading R5: the first step tries dt_0 = tau(S^0), which fails dt < tau
    stats, log, st = o.run(1e9, v.copy(), e.copy(), x.copy(), max_steps=1)
    assert stats["rejects"] >= 1
    assert log[0] <= 0.85 * tau0 * (1 + 1e-15)
    # a small step is accepted and the next proposal grows by beta2
    vv, ee, xx = v.copy(), e.copy(), x.copy()
    stats, log, st = o.run(1.0, vv, ee, xx, dt=1e-4, max_steps=1)
    assert stats["rejects"] == 0 and log[0] == 1e-4
    assert stats["dt"] == 1.02 * 1e-4


def test_dt_collapse_is_reported():
    # tau(S^0) ~ 0.042; from dt = 0.2 the redo cascade 0.2 * 0.85^n passes
    # below dt_min = 0.05 * t_final before any step is accepted
    o = _sedov(4, dt_min_frac=0.05)
    v, e, x = o.init_state()
    stats, _, st = o.run(1.0, v, e, x, dt=0.2)
    assert st == O.EDTMIN and stats["steps"] == 0 and stats["rejects"] == 9


def test_step_counts_sanity_band():
    """Not parity (the paper's counts come from Laghos on 3D meshes with its own
    viscosity): the 2D 8x8 blast to t = 0.8 takes a few hundred steps."""
    o = _sedov(8)
    v, e, x = o.init_state()
    stats, _, _ = o.run(0.8, v, e, x)
    assert 100 < stats["steps"] < 2000


@pytest.mark.parametrize("dim,k,lo,hi", [(2, 1, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)),
                                         (2, 3, (-0.5, -0.5, 0.0), (0.5, 1.5, 1.0)),
                                         (3, 2, (0.0, 0.0, 0.0), (2.0, 1.0, 0.5))])
def test_total_mass_closed_form(dim, k, lo, hi):
    """With rho0 = 1: 1.M_V.1 = d |Omega| (each component's basis sums to
    one) and 1.M_E.1 = |Omega|, on boxes that are not the unit square, so a
    Jacobian scale or a dropped quadrature weight shows."""
    o = O.Oracle(dim=dim, nx=3, ny=2, nz=2, order=k, problem=O.SEDOV, lo=list(lo), hi=list(hi))
    vol = float(np.prod([hi[i] - lo[i] for i in range(dim)]))
    one_v, one_e = np.ones(o.nv), np.ones(o.ne)
    assert abs(one_v @ o.mass_apply_v(one_v) - dim * vol) <= 1e-13 * dim * vol
    assert abs(one_e @ o.mass_apply_e(one_e) - vol) <= 1e-13 * vol
    # total energy of a uniform state: (|u|^2 / 2 + e) |Omega|
    u = np.array([0.3, -1.1, 0.7][:dim])
    v = np.repeat(u, o.nv // dim)
    E = o.total_energy(v, 2.5 * one_e)
    assert abs(E - (0.5 * u @ u + 2.5) * vol) <= 1e-13 * E


def test_taylor_green_half_turn_symmetry():
    """The Taylor-Green velocity, pressure and energy source are invariant under
    the half turn (x, y) -> (1 - x, 1 - y) of the unit square, which maps the
    velocity vector to minus itself.  So is the discrete state after steps with
    viscosity: node (i, j) -> (n-1-i, n-1-j), v -> -v, and each element's
    energy dofs reversed.  A reversed basis, a swapped index or a sign error in
    one direction breaks it."""
    n = 6
    o = O.Oracle(dim=2, nx=n, ny=n, order=2, problem=O.TAYLOR_GREEN, gamma=5.0 / 3.0, visc=1,
                 source=1, cfl=0.1)
    v, e, x = o.init_state()
    stats, _, st = o.run(0.05, v, e, x)
    assert st == O.OK and stats["steps"] > 10
    nn = 2 * n + 1
    V, X = v.reshape(2, nn, nn), x.reshape(2, nn, nn)  # [c][y][x]
    vmax = np.abs(V).max()
    assert vmax > 0.5
    assert np.abs(V[:, ::-1, ::-1] + V).max() <= 1e-11 * vmax
    assert np.abs(X[:, ::-1, ::-1] - (1.0 - X)).max() <= 1e-12
    E = e.reshape(n, n, 2, 2)  # [ey, ex, jy, jx]
    assert np.abs(E[::-1, ::-1, ::-1, ::-1] - E).max() <= 1e-11 * np.abs(e).max()
    # the swap x <-> y maps the flow to its time reversal, not to itself: the
    # energy after the steps is not swap-symmetric (the test tells them apart)
    assert np.abs(E - E.transpose(1, 0, 3, 2)).max() > 1e-9 * np.abs(e).max()


def test_gresho_quarter_turn_symmetry():
    """The vortex on the centred square is invariant under the quarter turn
    (x, y) -> (-y, x), which rotates the velocity vector: node (i, j) ->
    (n-1-j, i), v_x -> -v_y, v_y -> v_x."""
    n = 4
    o = O.Oracle(dim=2, nx=n, ny=n, order=3, problem=O.GRESHO, gamma=5.0 / 3.0, visc=0,
                 lo=[-0.5, -0.5, 0], hi=[0.5, 0.5, 1])
    v, e, x = o.init_state()
    stats, _, st = o.run(0.15, v, e, x)
    assert st == O.OK and stats["steps"] > 10
    nn = 3 * n + 1
    V = v.reshape(2, nn, nn)  # [c][y][x]
    vmax = np.abs(V).max()
    assert vmax > 0.5
    assert np.abs(V[0][:, ::-1].T + V[1]).max() <= 1e-11 * vmax
    assert np.abs(V[1][:, ::-1].T - V[0]).max() <= 1e-11 * vmax


def _element_density_and_radius(x, n):
    """Per element of an n x n Q2 mesh of the unit square (rho0 = 1): density
    as initial mass over the current area (polygon of the 8 boundary nodes),
    and the radius of the element's centre node."""
    nn = 2 * n + 1
    X, Y = x[:nn * nn].reshape(nn, nn), x[nn * nn:].reshape(nn, nn)
    ring = [(0, 0), (1, 0), (2, 0), (2, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    rho, rc = np.zeros((n, n)), np.zeros((n, n))
    for ey in range(n):
        for ex in range(n):
            px = np.array([X[2 * ey + j, 2 * ex + i] for i, j in ring])
            py = np.array([Y[2 * ey + j, 2 * ex + i] for i, j in ring])
            area = 0.5 * np.sum(px * np.roll(py, -1) - np.roll(px, -1) * py)
            rho[ey, ex] = (1.0 / n) ** 2 / area
            rc[ey, ex] = np.hypot(X[2 * ey + 1, 2 * ex + 1], Y[2 * ey + 1, 2 * ex + 1])
    return rho, rc


def test_sedov_shock_radius_matches_the_similarity_solution():
    """The blast of energy 0.25 in the corner of the reflecting quarter domain
    is the full-plane cylindrical blast of E = 1.  Sedov's similarity solution
    puts its shock at R = xi0 (E t^2 / rho0)^(1/4), xi0 = 1.004 for gamma = 1.4
    (textbook value, not from the paper): R(0.8) = 0.898.  On 16 x 16 Q2
    elements the front (where the density falls half-way back from its peak,
    along the wall) must lie within half an initial element width of it, and
    the peak compression below the strong-shock limit (gamma+1)/(gamma-1) = 6."""
    n = 16
    o = _sedov(n)
    v, e, x = o.init_state()
    stats, _, st = o.run(0.8, v, e, x)
    assert st == O.OK
    rho, rc = _element_density_and_radius(x, n)
    R = 1.004 * (1.0 * 0.8 ** 2 / 1.0) ** 0.25
    row, r = rho[0], rc[0]                      # the elements along the wall y = 0
    k = int(np.argmax(row))
    assert 3.0 < row[k] < 6.0
    half = 0.5 * (row[k] + 1.0)
    j = next(i for i in range(k, n - 1) if row[i] >= half > row[i + 1])
    front = r[j] + (row[j] - half) / (row[j] - row[j + 1]) * (r[j + 1] - r[j])
    assert abs(front - R) <= 0.5 / n
    # the unshocked gas ahead of the front is at rest at the initial density
    assert abs(row[-1] - 1.0) < 0.05
