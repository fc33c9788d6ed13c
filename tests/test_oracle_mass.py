"""Pins of the oracle's mass matrices M_V, M_E (eq:fom) and of its CG solve:
exact polynomial integration assembled independently, total mass, and a dense
Cholesky solve of the same system."""
import numpy as np
import pytest
from numpy.polynomial import polynomial as P

import oracle as O
from tests import _fem_ref as R


def _exact_1d_mass(nodes):
    polys = R.lagrange_polys(nodes)
    n = len(nodes)
    M = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            c = P.polyint(P.polymul(polys[a], polys[b]))
            M[a, b] = P.polyval(1.0, c) - P.polyval(0.0, c)
    return M


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(m, out)  # first index fastest
    return out


def _assemble_scalar(mesh, Mloc):
    M = np.zeros((mesh.nnodes, mesh.nnodes))
    for el in range(mesh.nelem):
        cn = mesh.conn(el)
        M[np.ix_(cn, cn)] += Mloc
    return M


@pytest.mark.parametrize("dim,n,k", [(2, (3, 2), 1), (2, (3, 2), 2), (2, (2, 2), 3),
                                     (3, (2, 2, 1), 2), (3, (1, 2, 1), 1)])
def test_mass_v_matches_exact_integration(dim, n, k):
    lo, hi = [0.0, -1.0, 0.5], [2.0, 0.5, 1.0]
    o = O.Oracle(dim=dim, nx=n[0], ny=n[1], nz=n[2] if dim == 3 else 1, order=k,
                 problem=O.UNIFORM, lo=lo, hi=hi)
    h = [(hi[c] - lo[c]) / n[c] for c in range(dim)]
    M1 = _exact_1d_mass(R.gauss_lobatto01(k + 1))
    Mloc = _kron_all([M1 * h[c] for c in range(dim)])
    mesh = R.CartesianMesh(dim, n, k)
    M = _assemble_scalar(mesh, Mloc)
    rng = np.random.default_rng(3)
    a = rng.normal(size=o.nv)
    got = o.mass_apply_v(a)
    want = np.concatenate([M @ a[c * o.nnodes:(c + 1) * o.nnodes] for c in range(dim)])
    assert np.allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())
    # 1^T M 1 per component = total mass = volume (rho0 = 1)
    vol = np.prod([hi[c] - lo[c] for c in range(dim)])
    ones = np.ones(o.nv)
    assert abs(ones @ o.mass_apply_v(ones) - dim * vol) < 1e-13 * dim * vol


@pytest.mark.parametrize("dim,n,k", [(2, (3, 2), 2), (2, (2, 2), 3), (3, (2, 1, 2), 2),
                                     (2, (2, 3), 1)])
def test_mass_e_matches_exact_integration(dim, n, k):
    o = O.Oracle(dim=dim, nx=n[0], ny=n[1], nz=n[2] if dim == 3 else 1, order=k,
                 problem=O.UNIFORM)
    h = [1.0 / n[c] for c in range(dim)]
    nodes = R.gauss_legendre01(k)[0] if k >= 1 else np.array([0.5])
    M1 = _exact_1d_mass(nodes)
    Mloc = _kron_all([M1 * h[c] for c in range(dim)])
    rng = np.random.default_rng(4)
    a = rng.normal(size=o.ne)
    got = o.mass_apply_e(a)
    want = (a.reshape(o.nelem, -1) @ Mloc.T).reshape(-1)
    assert np.allclose(got, want, atol=1e-15 * np.abs(want).max() * 10, rtol=0)
    back = o.mass_solve_e(got)
    assert np.allclose(back, a, atol=1e-12, rtol=0)
    assert abs(o.mass_apply_e(np.ones(o.ne)).sum() - 1.0) < 1e-14


@pytest.mark.parametrize("dim,n,k", [(2, (4, 3), 2), (2, (3, 3), 3), (3, (2, 2, 2), 2),
                                     (2, (5, 4), 1)])
def test_cg_matches_dense_cholesky(dim, n, k):
    o = O.Oracle(dim=dim, nx=n[0], ny=n[1], nz=n[2] if dim == 3 else 1, order=k,
                 problem=O.UNIFORM)
    rng = np.random.default_rng(5)
    b = rng.normal(size=o.nv)
    a_cg, its, relres, st = o.mass_solve_v(b)
    assert st == O.OK and relres <= 1e-14
    a_d = o.mass_solve_v_dense(b)
    assert np.linalg.norm(a_cg - a_d) <= 1e-13 * np.linalg.norm(a_d)
    ess = o.essential_mask()
    assert np.all(a_cg[ess] == 0.0)
    # the free rows of M a reproduce b
    r = o.mass_apply_v(a_cg) - b
    assert np.linalg.norm(r[~ess]) <= 1e-13 * np.linalg.norm(b)


def test_cg_zero_rhs_and_iteration_limit():
    o = O.Oracle(dim=2, nx=3, ny=3, order=2, problem=O.UNIFORM)
    a, its, relres, st = o.mass_solve_v(np.zeros(o.nv))
    assert st == O.OK and its == 0 and np.all(a == 0)
    o2 = O.Oracle(dim=2, nx=6, ny=6, order=2, problem=O.UNIFORM, cg_maxit=2)
    b = np.random.default_rng(0).normal(size=o2.nv)
    _, its, _, st = o2.mass_solve_v(b)
    assert st == O.ECG and its == 2
