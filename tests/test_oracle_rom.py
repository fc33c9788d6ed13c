"""Pins of the reference hyper-reduced step (oracle/rom.py; Section 3 with the
SNS bases of Section 4.2 and the DEIM sampling of Section 4.3).

DEIM: the sampled rows are distinct, the oblique projection reproduces every
vector of the basis span exactly, and its error obeys the bound of
eq:errorbound_DEIM with the constant ||(Z^T Phi)^+||.  The full-basis case
pins the whole step: with bases spanning every free degree of freedom and
every entry sampled, the hyper-reduced RK2-average step is the full-order
step (eq:RK2-avg-rom-hr reduces to eq:RK2-avg), the same accepted step sizes
included."""
import numpy as np
import pytest

import oracle as O
from oracle import rom


@pytest.mark.parametrize("N,m,ns", [(200, 8, 8), (200, 8, 20), (500, 25, 60), (40, 40, 40)])
def test_deim_interpolation_and_error_bound(N, m, ns):
    rng = np.random.default_rng(N + m + ns)
    Phi = np.linalg.qr(rng.normal(size=(N, m)))[0]
    p = rom.deim(Phi, ns)
    assert len(set(p.tolist())) == ns and p.min() >= 0 and p.max() < N
    A = np.linalg.pinv(Phi[p, :])
    assert np.allclose(A @ Phi[p, :], np.eye(m), atol=1e-11)
    kappa = np.linalg.norm(A, 2)
    for _ in range(5):
        f = rng.normal(size=N)
        err = np.linalg.norm(f - Phi @ (A @ f[p]))
        best = np.linalg.norm(f - Phi @ (Phi.T @ f))
        assert err <= kappa * best * (1 + 1e-10) + 1e-12


def test_deim_first_sample_is_the_largest_entry_and_ties_go_low():
    Phi = np.zeros((6, 1))
    Phi[[2, 4], 0] = [-3.0, 3.0]
    assert rom.deim(Phi, 1).tolist() == [2]
    assert rom.deim(Phi, 2 * 1).tolist() == [2, 4]


def _full_basis_rom(o):
    """Bases spanning every free degree of freedom, every entry sampled."""
    v0, e0, x0 = o.init_state()
    free = np.where(~o.essential_mask())[0]
    Iv = np.eye(o.nv)[:, free]
    Ie = np.eye(o.ne)
    pF = free.copy()
    pG = np.arange(o.ne)
    return rom.RomOracle(o, Iv, Ie, Iv.copy(), v0, e0, x0, pF, pG), v0, e0, x0, free


@pytest.mark.parametrize("problem,n", [(O.SEDOV, (3, 2)), (O.GRESHO, (2, 2))])
def test_full_basis_rom_is_the_full_order_step(problem, n):
    o = O.Oracle(dim=2, nx=n[0], ny=n[1], order=2, problem=problem,
                 lo=(-0.5, -0.5, 0) if problem == O.GRESHO else (0, 0, 0),
                 hi=(0.5, 0.5, 1) if problem == O.GRESHO else (1, 1, 1),
                 gamma=5.0 / 3.0 if problem == O.GRESHO else 1.4,
                 visc=0 if problem == O.GRESHO else 1)
    R, v0, e0, x0, free = _full_basis_rom(o)
    assert len(R.els) == o.nelem
    vh, eh, xh = np.zeros(len(free)), np.zeros(o.ne), np.zeros(len(free))
    v, e, x = v0.copy(), e0.copy(), x0.copy()
    for dt in (2e-3, 3e-3):
        vh, eh, xh, tau_r = R.step(dt, vh, eh, xh)
        tau_f, _, st = o.step(dt, v, e, x)
        assert st == O.OK and abs(tau_r - tau_f) <= 1e-14 * tau_f
        lv, le, lx = R.lift(vh, eh, xh)
        for a, b in ((v, lv), (e, le), (x, lx)):
            assert np.abs(a - b).max() <= 1e-11 * max(np.abs(a).max(), 1e-300)
    # the step control: the same accepted steps as the full-order loop
    vh, eh, xh = np.zeros(len(free)), np.zeros(o.ne), np.zeros(len(free))
    vh, eh, xh, t, dt, steps, rejects, log = R.run(0.05, vh, eh, xh)
    v, e, x = v0.copy(), e0.copy(), x0.copy()
    st, log_f, s = o.run(0.05, v, e, x)
    assert steps == st["steps"] and rejects == st["rejects"]
    assert np.allclose(log, log_f, rtol=1e-11, atol=0)
    lv, le, lx = R.lift(vh, eh, xh)
    assert np.abs(lv - v).max() <= 1e-10 * np.abs(v).max()
