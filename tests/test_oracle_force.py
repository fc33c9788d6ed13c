"""Pins of the oracle's force matrix F (eq:forceOneforceTv) and quadrature-point
physics (eq:EOS, eq:adaptive-timestep, viscosity reading R3).

The pressure part of F has closed forms that do not go through the oracle:
  * F.1 = -grad_x Phi with Phi(x) = (gamma-1) sum_q alpha_q rho0|J0|_q e_q ln|J_q(x)|
    (differentiating |J| gives adj(J)^T grad w_i), checked by complex-step
    differentiation of an independent numpy evaluation of |J_q(x)|;
  * (F^T v)_j = -sum_q alpha_q phi_j(q) p_q d/de |J_q(x + e v)|, likewise;
  * for a uniform gas at rest F.1 is the boundary integral -p \\oint w_i n_c.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as P

import oracle as O
from tests import _fem_ref as R


def _mesh_setup(dim, n, k, seed, amp=0.08):
    o = O.Oracle(dim=dim, nx=n[0], ny=n[1], nz=n[2] if dim == 3 else 1, order=k,
                 problem=O.UNIFORM, visc=0, gamma=1.4)
    v, e, x = o.init_state()
    rng = np.random.default_rng(seed)
    h = 1.0 / max(n)
    x = x + (amp / k) * h * rng.uniform(-1, 1, size=x.shape)
    e = rng.uniform(1.0, 2.0, size=e.shape)
    return o, v, e, x


def _tables(o):
    d, k = o.dim, o.cfg.order
    qp, qw = R.gauss_legendre01(o.cfg.nq)
    H, dH = R.tensor_basis(R.gauss_lobatto01(k + 1), qp, d)
    L, _ = R.tensor_basis(R.gauss_legendre01(k)[0], qp, d)
    alpha = R.tensor_weights(qw, d)
    mesh = R.CartesianMesh(d, [o.cfg.nx, o.cfg.ny, o.cfg.nz][:d], k)
    return H, dH, L, alpha, mesh


def _detJ_all(o, x, tabs):
    H, dH, L, alpha, mesh = tabs
    d = o.dim
    out = []
    for el in range(mesh.nelem):
        cn = mesh.conn(el)
        xl = np.stack([x[c * o.nnodes + cn] for c in range(d)])  # [c, i]
        J = np.einsum("ci,qim->qcm", xl, dH)
        out.append(np.linalg.det(J) if not np.iscomplexobj(J) else _cdet(J))
    return np.array(out)  # [el, q]


def _cdet(J):
    if J.shape[-1] == 2:
        return J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    return (J[:, 0, 0] * (J[:, 1, 1] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 1])
            - J[:, 0, 1] * (J[:, 1, 0] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 0])
            + J[:, 0, 2] * (J[:, 1, 0] * J[:, 2, 1] - J[:, 1, 1] * J[:, 2, 0]))


def _F1_unconstrained(o, v, e, x):
    d = o.dim
    F1 = np.zeros(o.nv)
    mesh = R.CartesianMesh(d, [o.cfg.nx, o.cfg.ny, o.cfg.nz][:d], o.cfg.order)
    for el in range(o.nelem):
        FK = o.element_force_matrix(el, v, e, x)
        rows = FK.sum(axis=1).reshape(d, o.nd1)
        cn = mesh.conn(el)
        for c in range(d):
            np.add.at(F1, c * o.nnodes + cn, rows[c])
    return F1


@pytest.mark.parametrize("dim,n,k", [(2, (3, 2), 2), (2, (2, 2), 3), (3, (2, 1, 1), 2),
                                     (2, (2, 3), 1)])
def test_F1_is_minus_gradient_of_pressure_potential(dim, n, k):
    o, v, e, x = _mesh_setup(dim, n, k, seed=11)
    tabs = _tables(o)
    H, dH, L, alpha, mesh = tabs
    vol = np.prod([1.0 / m for m in n])
    eq = (e.reshape(o.nelem, -1) @ L.T)  # [el, q]
    w = (o.cfg.gamma - 1.0) * vol * alpha[None, :] * eq

    def phi(xx):
        return np.sum(w * np.log(_detJ_all(o, xx, tabs)))

    grad = np.zeros(o.nv)
    hstep = 1e-30
    for i in range(o.nv):
        xc = x.astype(np.complex128)
        xc[i] += 1j * hstep
        grad[i] = phi(xc).imag / hstep
    F1 = _F1_unconstrained(o, v, e, x)
    assert np.allclose(F1, -grad, rtol=0, atol=1e-12 * np.abs(grad).max())
    # with boundary conditions the essential components are zero, others equal
    F1bc, _, _, st = o.force(v, e, x)
    ess = o.essential_mask()
    assert st == O.OK
    assert np.all(F1bc[ess] == 0.0)
    assert np.allclose(F1bc[~ess], -grad[~ess], rtol=0, atol=1e-12 * np.abs(grad).max())


@pytest.mark.parametrize("dim,n,k", [(2, (3, 2), 2), (3, (1, 2, 1), 2), (2, (2, 2), 3)])
def test_FTv_is_pressure_work(dim, n, k):
    o, _, e, x = _mesh_setup(dim, n, k, seed=12)
    tabs = _tables(o)
    H, dH, L, alpha, mesh = tabs
    rng = np.random.default_rng(13)
    vt = rng.normal(size=o.nv)
    vol = np.prod([1.0 / m for m in n])
    eq = (e.reshape(o.nelem, -1) @ L.T)
    det0 = _detJ_all(o, x, tabs)
    p = (o.cfg.gamma - 1.0) * vol * eq / det0
    hstep = 1e-30
    ddet = _detJ_all(o, x.astype(np.complex128) + 1j * hstep * vt, tabs).imag / hstep
    want = -np.einsum("q,eq,eq,qj->ej", alpha, p, ddet, L).reshape(-1)
    _, FTv, _, st = o.force(np.zeros(o.nv), e, x, vtest=vt)
    assert st == O.OK
    assert np.allclose(FTv, want, rtol=0, atol=1e-12 * np.abs(want).max())


def _int01(poly):
    c = P.polyint(poly)
    return P.polyval(1.0, c) - P.polyval(0.0, c)


@pytest.mark.parametrize("dim,n,k", [(2, (3, 2), 2), (2, (2, 2), 3), (3, (2, 2, 1), 2)])
def test_uniform_gas_force_is_boundary_integral(dim, n, k):
    e0, gam = 1.7, 1.4
    o = O.Oracle(dim=dim, nx=n[0], ny=n[1], nz=n[2] if dim == 3 else 1, order=k,
                 problem=O.UNIFORM, e_uniform=e0, gamma=gam, visc=1)
    v, e, x = o.init_state()
    p = (gam - 1.0) * 1.0 * e0
    F1 = _F1_unconstrained(o, v, e, x)
    # int_0^1 of each 1D GLL Lagrange polynomial
    w1 = np.array([_int01(c) for c in R.lagrange_polys(R.gauss_lobatto01(k + 1))])
    nn = [m * k + 1 for m in n]
    h = [1.0 / m for m in n]
    # 1D integral of the global hat function of node I along one direction
    def hat_int(I, c):
        a = I % k
        val = 0.0
        if I < nn[c] - 1:
            val += w1[a] * h[c]
        if a == 0 and I > 0:
            val += w1[k] * h[c]
        return val
    want = np.zeros(o.nv)
    for node in range(o.nnodes):
        I = [(node // int(np.prod(nn[:c]))) % nn[c] for c in range(dim)]
        for c in range(dim):
            if I[c] not in (0, nn[c] - 1):
                continue
            nrm = 1.0 if I[c] == nn[c] - 1 else -1.0
            face = np.prod([hat_int(I[m], m) for m in range(dim) if m != c])
            want[c * o.nnodes + node] = -p * nrm * face
    assert np.allclose(F1, want, rtol=0, atol=1e-13 * p)
    # after the wall condition nothing is left: the gas stays at rest
    F1bc, _, dt, _ = o.force(v, e, x)
    assert np.abs(F1bc).max() < 1e-14 * p
    # closed-form estimate: tau = alpha h_min / c_s with h_min = h/k
    cs = np.sqrt(gam * (gam - 1.0) * e0)
    assert abs(dt - 0.5 * (min(h) / k) / cs) < 1e-15


def _qp_oracle(dim, k=2, nel=8, **kw):
    return O.Oracle(dim=dim, nx=nel, ny=nel, nz=nel if dim == 3 else 1, order=k,
                    problem=O.UNIFORM, **kw)


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.1])
def test_qpoint_uniaxial_compression_closed_form(theta):
    o = _qp_oracle(2, gamma=1.4, visc=1)
    h, k, lam, e_q = 1.0 / 8, 2, 3.0, 2.0
    R_ = np.array([[np.cos(theta), -np.sin(theta)], [np.sin(theta), np.cos(theta)]])
    J = R_ @ np.diag([h, h])                     # rotated element, |J| = h^2
    nvec = R_[:, 0]
    gradv = -lam * np.outer(nvec, nvec)          # compression along n
    sigma, tau, mu, st = o.qpoint(J, gradv @ J, e_q, h * h)
    assert st == O.OK
    rho, p = 1.0, 0.4 * 2.0
    cs = np.sqrt(1.4 * 0.4 * e_q)
    ell = h / k                                  # |J J0^-1 n| = |R n| = 1
    mu_want = rho * (2.0 * ell ** 2 * lam + 0.5 * ell * cs)
    assert abs(mu - mu_want) < 1e-14 * mu_want
    assert np.allclose(sigma, -p * np.eye(2) - mu_want * lam * np.outer(nvec, nvec), atol=1e-13)
    hmin = h / k
    tau_want = 0.5 / (cs / hmin + 2.5 * mu_want / (rho * hmin ** 2))
    assert abs(tau - tau_want) < 1e-14 * tau_want


def test_qpoint_stretched_element_length_scales():
    o = _qp_oracle(2, gamma=1.4, visc=1)
    h, k, lam, e_q = 1.0 / 8, 2, 1.5, 1.0
    J = np.diag([2 * h, h])                      # stretched twice along x
    gradv = np.diag([-lam, 0.0])
    sigma, tau, mu, st = o.qpoint(J, gradv @ J, e_q, h * h)
    rho = 0.5                                    # volume doubled
    cs = np.sqrt(1.4 * 0.4 * e_q)
    ell = 2 * h / k                              # l_0 |J J0^-1 e_x| = 2 l_0
    mu_want = rho * (2.0 * ell ** 2 * lam + 0.5 * ell * cs)
    assert abs(mu - mu_want) < 1e-14 * mu_want
    hmin = h / k                                 # sigma_min(J) / k
    tau_want = 0.5 / (cs / hmin + 2.5 * mu_want / (rho * hmin ** 2))
    assert abs(tau - tau_want) < 1e-14 * tau_want
    p = 0.4 * rho * e_q
    assert np.allclose(sigma, np.diag([-p - mu_want * lam, -p]), atol=1e-14)


def test_qpoint_expansion_has_no_viscosity_and_3d_direction():
    o = _qp_oracle(2, gamma=5.0 / 3.0, visc=1)
    h = 1.0 / 8
    J = np.diag([h, h])
    sigma, tau, mu, _ = o.qpoint(J, np.diag([0.7, 0.2]) @ J, 3.0, h * h)
    assert mu == 0.0
    p = (2.0 / 3.0) * 3.0
    assert np.allclose(sigma, -p * np.eye(2), atol=1e-15)
    cs = np.sqrt((5.0 / 3.0) * (2.0 / 3.0) * 3.0)
    assert abs(tau - 0.5 * (h / 2) / cs) < 1e-15
    o3 = _qp_oracle(3, gamma=1.4, visc=1, nel=4)
    h3 = 0.25
    J3 = np.diag([h3, 2 * h3, h3])
    gradv = np.diag([0.1, -2.0, 0.3])
    sigma, tau, mu, _ = o3.qpoint(J3, gradv @ J3, 1.0, h3 ** 3)
    rho = 0.5
    ell = 2 * h3 / 2                              # compression along y, stretched 2x
    cs = np.sqrt(1.4 * 0.4)
    mu_want = rho * (2.0 * ell ** 2 * 2.0 + 0.5 * ell * cs)
    assert abs(mu - mu_want) < 1e-13 * mu_want


def test_qpoint_tangled_and_negative_energy():
    o = _qp_oracle(2, visc=1)
    _, tau, _, st = o.qpoint(np.array([[0.1, 0.0], [0.0, -0.1]]), np.zeros((2, 2)), 1.0, 0.01)
    assert st == O.ETANGLED and tau == 0.0
    sigma, tau, mu, st = o.qpoint(np.eye(2) * 0.1, np.zeros((2, 2)), -1.0, 0.01)
    assert st == O.OK and np.isinf(tau) and mu == 0.0
    assert sigma[0, 0] == pytest.approx(0.4)     # p = (gamma-1) rho e < 0


def test_energy_identity_with_viscosity():
    o = O.Oracle(dim=2, nx=4, ny=3, order=2, problem=O.UNIFORM, visc=1)
    v, e, x = o.init_state()
    rng = np.random.default_rng(21)
    x = x + 0.05 * 0.25 * rng.uniform(-1, 1, size=x.shape)
    e = rng.uniform(0.5, 2.0, size=e.shape)
    v = rng.normal(size=v.shape)
    v[o.essential_mask()] = 0.0
    F1, FTv, dt, st = o.force(v, e, x, vtest=v)
    assert st == O.OK and dt > 0
    assert abs(v @ F1 - FTv.sum()) < 1e-13 * np.abs(v).max() * np.abs(F1).sum()


def test_sedov_initial_estimate_closed_form():
    o = O.Oracle(dim=2, nx=8, ny=8, order=2, problem=O.SEDOV)
    v, e, x = o.init_state()
    e0 = 0.25 / (1.0 / 64)
    assert np.all(e[:4] == e0) and np.all(e[4:] == 0.0)
    _, _, dt, st = o.force(v, e, x)
    cs = np.sqrt(1.4 * 0.4 * e0)
    assert st == O.OK and abs(dt - 0.5 * (1.0 / 16) / cs) < 1e-16
