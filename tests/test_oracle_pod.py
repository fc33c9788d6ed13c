"""Pins of the oracle's offline stage (Section 4): snapshot collection with
the intermediate RK2-average stage, the thin SVD of eq:SVD by one-sided
Jacobi, and the POD basis with the energy criterion of eq:energy_criteria.

The SVD is checked against numpy.linalg.svd (an independent LAPACK routine):
singular values and left singular vectors up to sign.  The basis properties
hold for any correct thin SVD: orthonormal columns, the residual of the rank-k
projection equal to the discarded singular values (||S - U_k U_k^T S||_F^2 =
sum_{i>k} sigma_i^2), and the smallest k that meets the criterion.  The
snapshot columns are checked against the oracle's own step taken one at a
time: column 2j+1 is the state after step j+1, column 2j the half-step state
S^{n+1/2} of that step, rebuilt from the force and mass solves."""
import numpy as np
import pytest

import oracle as O


def _mat(m, n, rank, seed, decay=0.3):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, rank)) @ np.diag(np.exp(-decay * np.arange(rank))) @ rng.normal(size=(rank, n))
    return A


@pytest.mark.parametrize("m,n,rank", [(40, 12, 12), (200, 30, 9), (57, 57, 57), (30, 45, 30)])
def test_jacobi_svd_matches_lapack(m, n, rank):
    A = _mat(m, n, rank, seed=m + n)
    US, sg, sweeps, st = O.svd_jacobi(A)
    assert st == O.OK and sweeps < 30
    order = np.argsort(-sg)
    s_ref = np.linalg.svd(A, compute_uv=False)
    kk = min(m, n)
    assert np.allclose(sg[order][:kk], s_ref, rtol=0, atol=1e-13 * s_ref[0])
    U_ref = np.linalg.svd(A, full_matrices=False)[0]
    # left vectors of the well-separated leading values, up to sign
    for r in range(min(rank, kk) - 1):
        gap = min(abs(s_ref[r] - s_ref[r + 1]), abs(s_ref[r] - s_ref[r - 1]) if r else np.inf)
        if gap < 1e-3 * s_ref[0]:
            continue
        u = US[order[r]] / sg[order[r]]
        assert min(np.abs(u - U_ref[:, r]).max(), np.abs(u + U_ref[:, r]).max()) < 1e-10
    # U Sigma W^T = A: the rotated columns span A's column space isometrically
    assert abs(np.sum(sg ** 2) - np.sum(A * A)) < 1e-12 * np.sum(A * A)


@pytest.mark.parametrize("eps", [0.9999, 0.99, 0.9])
def test_pod_basis_properties(eps):
    m, n = 120, 40
    S = _mat(m, n, 25, seed=7, decay=0.5)
    off = np.linspace(-1.0, 1.0, m)
    S_cols = (S + off[:, None]).T.copy()            # snapshots as columns, with an offset
    U, sg, k, st = O.pod(S_cols, offset=off, eps=eps)
    assert st == O.OK
    assert np.all(np.diff(sg) <= 0)
    s_ref = np.linalg.svd(S, compute_uv=False)
    assert np.allclose(sg[:len(s_ref)], s_ref, atol=1e-13 * s_ref[0])
    Uk = U[:k].T
    assert np.allclose(Uk.T @ Uk, np.eye(k), atol=1e-13)
    res = S - Uk @ (Uk.T @ S)
    assert abs(np.sum(res * res) - np.sum(sg[k:] ** 2)) < 1e-10 * np.sum(sg ** 2)
    csum = np.cumsum(sg) / np.sum(sg)
    assert csum[k - 1] >= eps and (k == 1 or csum[k - 2] < eps)


def test_pod_of_zero_matrix_and_rank_one():
    U, sg, k, st = O.pod(np.zeros((5, 8)))
    assert k == 0 and np.all(sg == 0)
    a = np.arange(1.0, 9.0)
    U, sg, k, st = O.pod(np.outer([1.0, -2.0, 0.5], a))
    assert k == 1
    assert abs(sg[0] - np.linalg.norm(a) * np.linalg.norm([1.0, -2.0, 0.5])) < 1e-13 * sg[0]
    u = U[0]
    assert min(np.abs(u - a / np.linalg.norm(a)).max(), np.abs(u + a / np.linalg.norm(a)).max()) < 1e-14


def test_snapshots_are_the_stage_states():
    o = O.Oracle(dim=2, nx=6, ny=6, order=2, problem=O.SEDOV)
    v, e, x = o.init_state()
    stats, Sv, Se, Sx, st = o.run_snapshots(0.05, v, e, x, cap=400)
    assert st == O.OK and stats["snapshots"] == 2 * stats["steps"] and stats["steps"] > 3
    assert np.array_equal(Sv[-1], v) and np.array_equal(Se[-1], e) and np.array_equal(Sx[-1], x)
    # replay one step at a time
    w = o.init_state()
    _, log, _ = o.run(0.05, *[a.copy() for a in w])
    v1, e1, x1 = w
    for j, dt in enumerate(log):
        F1, _, _, _ = o.force(v1, e1, x1)
        a = o.mass_solve_v(-F1)[0]
        vh = v1 + 0.5 * dt * a
        _, FTv, _, _ = o.force(v1, e1, x1, vtest=vh)
        eh = e1 + 0.5 * dt * o.mass_solve_e(FTv)
        xh = x1 + 0.5 * dt * vh
        for got, want in ((Sv[2 * j], vh), (Se[2 * j], eh), (Sx[2 * j], xh)):
            assert np.abs(got - want).max() <= 1e-13 * max(1.0, np.abs(want).max())
        o.step(float(dt), v1, e1, x1)
        assert np.array_equal(Sv[2 * j + 1], v1) and np.array_equal(Se[2 * j + 1], e1)
        assert np.array_equal(Sx[2 * j + 1], x1)
