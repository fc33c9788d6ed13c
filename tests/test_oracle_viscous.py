"""Pin of the oracle's element force matrix with an anisotropic stress
(eq:forceOneforceTv with the viscous stress sigma_a of eq:euler, reading R3).

With sigma = -p I the products sigma adj(J)^T and adj(J)^T sigma coincide, so
the pressure pins cannot see a transposed or swapped stress contraction.  Here
the element matrix is rebuilt from its definition,

    F_K[(i,c), j] = int_K sigma : grad w_(i,c) phi_j dx
                  = sum_q alpha_q |J_q| phi_j(q) sum_n sigma_q[c,n] (grad_x w_i)_n,

in numpy, with physical gradients grad_ref w J^{-1} from numpy.linalg.inv and
the volume weight |J_q| alpha_q, on distorted elements under a compressive
velocity field (viscosity active, sigma anisotropic).  The stress is taken two
ways: from the oracle's quadrature-point routine (itself pinned by closed forms
in test_oracle_force.py), and from an independent numpy evaluation of reading
R3 (numpy.linalg.eigh for the smallest strain-rate eigenpair).  A last test
plants the swapped product in a scratch copy of the oracle source and checks
that the pin fails on it.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from tests import _fem_ref as R

CASES = [(2, (2, 2), 1), (2, (2, 1), 2), (2, (1, 2), 3), (3, (1, 1, 1), 1), (3, (2, 1, 1), 2)]


def _setup(dim, n, k, seed):
    o = O.Oracle(dim=dim, nx=n[0], ny=n[1], nz=n[2] if dim == 3 else 1, order=k,
                 problem=O.UNIFORM, visc=1, gamma=1.4)
    _, _, x0 = o.init_state()
    rng = np.random.default_rng(seed)
    h = 1.0 / max(n)
    x = x0 + (0.12 / k) * h * rng.uniform(-1, 1, size=x0.shape)
    nn = o.nnodes
    # compression towards an off-centre point, sheared, plus noise: the
    # strain rate has a negative eigenvalue at every point, in no fixed axis
    ctr = np.array([0.41, 0.57, 0.46])[:dim]
    X = x0.reshape(dim, nn)
    A = np.array([[-3.0, 1.3, 0.4], [-0.7, -1.1, 0.9], [0.5, -0.6, -2.2]])[:dim, :dim]
    v = (A @ (X - ctr[:, None])).reshape(-1) + 0.2 * rng.normal(size=dim * nn)
    e = rng.uniform(0.5, 2.0, size=o.ne)
    return o, v, e, x


def _tables(o):
    d, k = o.dim, o.cfg.order
    qp, qw = R.gauss_legendre01(o.cfg.nq)
    H, dH = R.tensor_basis(R.gauss_lobatto01(k + 1), qp, d)
    L, _ = R.tensor_basis(R.gauss_legendre01(k)[0], qp, d)
    alpha = R.tensor_weights(qw, d)
    mesh = R.CartesianMesh(d, [o.cfg.nx, o.cfg.ny, o.cfg.nz][:d], k)
    return dH, L, alpha, mesh


def _element_fields(o, el, v, e, x, tabs):
    dH, L, alpha, mesh = tabs
    d = o.dim
    cn = mesh.conn(el)
    xl = np.stack([x[c * o.nnodes + cn] for c in range(d)])
    vl = np.stack([v[c * o.nnodes + cn] for c in range(d)])
    J = np.einsum("ci,qim->qcm", xl, dH)
    Gv = np.einsum("ci,qim->qcm", vl, dH)
    eq = L @ e[el * o.nd2:(el + 1) * o.nd2]
    return J, Gv, eq


def _sigma_numpy(o, J, Gv, e_q, vol):
    """Reading R3 evaluated independently: rho from mass conservation, ideal
    gas pressure, eps = sym(grad v) with grad v = Gv J^{-1}, the smallest
    eigenpair by numpy.linalg.eigh, l_s = l_0 |J J0^{-1} s| on the initial
    Cartesian element, mu = rho (q2 l_s^2 |lambda| + q1 l_s c_s)."""
    d = o.dim
    gam, q1, q2, k = o.cfg.gamma, o.cfg.q1, o.cfg.q2, o.cfg.order
    h0 = np.array([(o.cfg.hi[c] - o.cfg.lo[c]) / [o.cfg.nx, o.cfg.ny, o.cfg.nz][c]
                   for c in range(d)])
    detJ = np.linalg.det(J)
    rho = vol / detJ
    p = (gam - 1.0) * rho * e_q
    cs = np.sqrt(max(0.0, gam * (gam - 1.0) * e_q))
    gv = Gv @ np.linalg.inv(J)
    eps = 0.5 * (gv + gv.T)
    lam, vecs = np.linalg.eigh(eps)
    sig = -p * np.eye(d)
    mu = 0.0
    hmin = np.linalg.svd(J, compute_uv=False).min() / k
    if lam[0] < -1e-5 * (np.linalg.norm(eps) + cs / hmin):
        s = vecs[:, 0]
        ell = (np.prod(h0) ** (1.0 / d) / k) * np.linalg.norm(J @ (s / h0))
        mu = rho * (q2 * ell * ell * abs(lam[0]) + q1 * ell * cs)
        sig = sig + mu * eps
    return sig, mu


def _FK_numpy(o, el, v, e, x, tabs, sigma_of):
    """F_K from its integral definition: (rows c * ndof_h1 + i, columns j)."""
    dH, L, alpha, mesh = tabs
    d = o.dim
    J, Gv, eq = _element_fields(o, el, v, e, x, tabs)
    FK = np.zeros((d, o.nd1, o.nd2))
    mus = []
    for q in range(len(alpha)):
        sig, mu = sigma_of(J[q], Gv[q], eq[q])
        mus.append(mu)
        Jinv = np.linalg.inv(J[q])
        gradw = dH[q] @ Jinv                       # [i, n] physical gradient of w_i
        dx = alpha[q] * np.linalg.det(J[q])        # volume weight
        integrand = np.einsum("cn,in->ci", sig, gradw)  # sigma : grad w_(i,c)
        FK += dx * integrand[:, :, None] * L[q][None, None, :]
    return FK.reshape(d * o.nd1, o.nd2), np.array(mus)


def _vol(o):
    return np.prod([(o.cfg.hi[c] - o.cfg.lo[c]) / [o.cfg.nx, o.cfg.ny, o.cfg.nz][c]
                    for c in range(o.dim)])


@pytest.mark.parametrize("dim,n,k", CASES)
def test_viscous_element_force_matrix_from_definition(dim, n, k):
    o, v, e, x = _setup(dim, n, k, seed=31 + 7 * k + dim)
    tabs = _tables(o)
    vol = _vol(o)

    def sigma_oracle(J, Gv, e_q):
        sig, _, mu, st = o.qpoint(J, Gv, e_q, vol)
        assert st == O.OK
        return sig, mu

    def sigma_indep(J, Gv, e_q):
        return _sigma_numpy(o, J, Gv, e_q, vol)

    for el in range(o.nelem):
        FK = o.element_force_matrix(el, v, e, x)
        want, mus = _FK_numpy(o, el, v, e, x, tabs, sigma_oracle)
        # the case exercises the viscous branch: mu > 0 at every point, and the
        # viscous part is not small against the pressure part
        assert np.all(mus > 0.0)
        scale = np.abs(want).max()
        assert np.abs(FK - want).max() <= 1e-13 * scale
        want2, mus2 = _FK_numpy(o, el, v, e, x, tabs, sigma_indep)
        assert np.allclose(mus2, mus, rtol=1e-12, atol=0)
        assert np.abs(FK - want2).max() <= 1e-12 * scale


@pytest.mark.parametrize("dim,n,k", [(2, (2, 1), 2), (3, (1, 1, 1), 2)])
def test_viscous_part_is_anisotropic(dim, n, k):
    """The stress of these cases is far from a multiple of the identity, so a
    swapped sigma adj(J)^T product changes F_K by much more than rounding."""
    o, v, e, x = _setup(dim, n, k, seed=5)
    tabs = _tables(o)
    vol = _vol(o)
    J, Gv, eq = _element_fields(o, 0, v, e, x, tabs)
    worst = 0.0
    for q in range(len(eq)):
        sig, _, mu, _ = o.qpoint(J[q], Gv[q], eq[q], vol)
        A = np.linalg.det(J[q]) * np.linalg.inv(J[q])   # adj(J)
        d1 = sig @ A.T
        d2 = A.T @ sig
        worst = max(worst, np.abs(d1 - d2).max() / np.abs(d1).max())
    assert worst > 1e-2


def _mutant_lib(tmp_path):
    """The oracle source with the stress contraction D = sigma adj(J)^T
    replaced by adj(J)^T sigma (a plausible index mistake), compiled apart."""
    src = open(os.path.join(os.path.dirname(O.__file__), "lagh_oracle.c")).read()
    good = "for (int n = 0; n < d; ++n) acc += sigma[c * d + n] * A[m * d + n];"
    bad = "for (int n = 0; n < d; ++n) acc += A[n * d + c] * sigma[n * d + m];"
    assert src.count(good) == 1
    mut = tmp_path / "lagh_oracle_mutant.c"
    mut.write_text(src.replace(good, bad))
    hdr = os.path.join(os.path.dirname(O.__file__), "lagh_oracle.h")
    (tmp_path / "lagh_oracle.h").write_text(open(hdr).read())
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(mut), "-lm"])
    L = ctypes.CDLL(str(so))
    L.lho_create.restype = ctypes.c_void_p
    L.lho_create.argtypes = [ctypes.POINTER(O._Config)]
    L.lho_destroy.argtypes = [ctypes.c_void_p]
    L.lho_element_force_matrix.argtypes = [ctypes.c_void_p, ctypes.c_long] + [O._dp] * 4
    return L


def test_pin_detects_swapped_stress_contraction(tmp_path):
    if subprocess.call(["gcc", "--version"], stdout=subprocess.DEVNULL) != 0:
        pytest.skip("no C compiler")
    L = _mutant_lib(tmp_path)
    for dim, n, k in [(2, (2, 1), 2), (3, (1, 1, 1), 2)]:
        o, v, e, x = _setup(dim, n, k, seed=31 + 7 * k + dim)
        tabs = _tables(o)
        vol = _vol(o)
        h = L.lho_create(ctypes.byref(o.cfg))
        assert h
        try:
            FK = np.zeros((dim * o.nd1, o.nd2))
            st = L.lho_element_force_matrix(h, 0, O._p(v), O._p(e), O._p(x), O._p(FK))
            assert st == O.OK
        finally:
            L.lho_destroy(h)
        want, _ = _FK_numpy(o, 0, v, e, x, tabs, lambda J, Gv, q: _sigma_numpy(o, J, Gv, q, vol))
        # the real oracle passes the pin (above); the mutant fails it by far
        assert np.abs(FK - want).max() > 1e-3 * np.abs(want).max()
