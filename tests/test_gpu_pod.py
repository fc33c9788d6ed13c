"""Offline stage on the GPU (Section 4): snapshot capture in the batched run
and the POD basis (eq:SVD, eq:energy_criteria), against the oracle.

Snapshots: for every accepted step the stage state S^{n+1/2} and then
S^{n+1}; each captured column is compared element by element with the
oracle's snapshot collector on the same instance (FP64 run).  POD: the GPU's
parallel one-sided Jacobi against the oracle's cyclic one on the same matrix
(singular values, the basis size of the criterion, leading vectors up to sign,
orthonormality), and the basis of the GPU snapshots against the oracle's basis
of its own snapshots."""
import numpy as np
import pytest

import oracle as O
from paper_2104_11404_gb300 import workloads as W
from tests._pair import oracle_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gpu_pod(S_cols, offset=None, eps=0.9999):
    from paper_2104_11404_gb300 import lagh
    S = torch.from_numpy(np.ascontiguousarray(S_cols)).cuda()
    n, m = S_cols.shape
    U = torch.zeros(n * m, dtype=torch.float64, device="cuda")
    sig = torch.zeros(n, dtype=torch.float64, device="cuda")
    work = torch.zeros(m * n + 2 * n + 16, dtype=torch.float64, device="cuda")
    off = None if offset is None else torch.from_numpy(np.ascontiguousarray(offset)).cuda()
    k, sweeps = lagh.lh_pod(S, m, n, off, eps, U, sig, work,
                            torch.cuda.current_stream().cuda_stream)
    return U.view(n, m).cpu().numpy(), sig.cpu().numpy(), k, sweeps


def _same_up_to_sign(a, b):
    return min(np.abs(a - b).max(), np.abs(a + b).max())


def _check_pod_pair(Ug, sg, kg, Uo, so, ko, sep=1e-3, vec_tol=1e-9):
    assert kg == ko
    assert np.abs(sg - so).max() <= 1e-12 * max(so[0], 1e-300) + 1e-300
    Uk = Ug[:kg].T
    assert np.abs(Uk.T @ Uk - np.eye(kg)).max() <= 1e-12
    for r in range(kg):
        lo = abs(so[r] - so[r + 1]) if r + 1 < len(so) else np.inf
        hi = abs(so[r] - so[r - 1]) if r > 0 else np.inf
        if min(lo, hi) < sep * so[0]:
            continue
        assert _same_up_to_sign(Ug[r], Uo[r]) <= vec_tol


@pytest.mark.parametrize("m,n,rank", [(300, 40, 40), (1000, 64, 20), (50, 80, 50), (64, 1, 1)])
def test_pod_matches_oracle(m, n, rank):
    rng = np.random.default_rng(m * n)
    A = (rng.normal(size=(m, rank)) @ np.diag(np.exp(-0.4 * np.arange(rank))) @
         rng.normal(size=(rank, n)))
    off = rng.normal(size=m)
    S_cols = (A + off[:, None]).T.copy()
    Ug, sg, kg, sweeps = _gpu_pod(S_cols, off)
    Uo, so, ko, st = O.pod(S_cols, off)
    assert st == O.OK and sweeps < 30
    _check_pod_pair(Ug, sg, kg, Uo, so, ko)


def _sedov(n, gamma=1.4, e0=0.25):
    return dict(dim=2, n=(n[0], n[1], 1), order=2, problem=W.SEDOV, gamma=gamma,
                lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1, blast_energy=e0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_batch_snapshots_match_oracle(precision, tol):
    from paper_2104_11404_gb300.batch import Batch
    cfgs = [_sedov((6, 6)), _sedov((8, 7), 1.6, 0.6), _sedov((5, 5), 1.35, 0.15)]
    t_final, cap = 0.05, 400
    b = Batch(cfgs, precision=precision)
    b.init_state()
    Sv, Se, Sx = b.snapshots([0, 2], cap)
    b.run_to(t_final)
    views = b.snapshot_views(Sv, Se, Sx)
    q = b.query()
    for i, cnt, V, E, X in views:
        assert cnt == 2 * q["steps"][i] and cnt > 6
        o = oracle_for(cfgs[i])
        v, e, x = o.init_state()
        st, Ov, Oe, Ox, s = o.run_snapshots(t_final, v, e, x, cap)
        assert s == O.OK and st["snapshots"] == cnt
        for got, want in ((V, Ov), (E, Oe), (X, Ox)):
            got = got.cpu().numpy()
            for c in range(cnt):
                scale = max(np.abs(want[c]).max(), 1e-300)
                assert np.abs(got[c] - want[c]).max() <= tol * scale, (i, c)
    b.close()


def test_pod_of_batch_snapshots_matches_oracle():
    from paper_2104_11404_gb300.batch import Batch
    cfg = _sedov((8, 8))
    t_final, cap = 0.1, 600
    b = Batch([cfg], precision="fp64")
    b.init_state()
    v0, e0, x0 = (t.clone() for t in b.get_state())
    Sv, Se, Sx = b.snapshots([0], cap)
    b.run_to(t_final)
    (_, cnt, V, E, X), = b.snapshot_views(Sv, Se, Sx)
    o = oracle_for(cfg)
    v, e, x = o.init_state()
    _, Ov, Oe, Ox, s = o.run_snapshots(t_final, v, e, x, cap)
    assert s == O.OK and len(Ov) == cnt
    vi, ei, xi = o.init_state()
    for gpu_cols, orc_cols, off_g, off_o in ((V, Ov, v0, vi), (E, Oe, e0, ei), (X, Ox, x0, xi)):
        Ug, sg, kg, _ = _gpu_pod(gpu_cols.cpu().numpy(), off_g.cpu().numpy())
        Uo, so, ko, st = O.pod(orc_cols, off_o)
        assert st == O.OK and kg >= 1
        assert kg == ko
        assert np.abs(sg[:kg] - so[:kg]).max() <= 1e-8 * so[0]
        for r in range(min(kg, 3)):
            if abs(so[r] - so[r + 1]) > 1e-2 * so[0] and (r == 0 or abs(so[r] - so[r - 1]) > 1e-2 * so[0]):
                assert _same_up_to_sign(Ug[r], Uo[r]) <= 1e-6
    b.close()
