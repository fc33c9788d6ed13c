"""Hyper-reduced online step on the GPU (Section 3, eq:RK2-avg-rom-hr, with
the SNS bases of Section 4.2 and DEIM sampling of Section 4.3) against the
oracle's plain reference (oracle/rom.py).

Full-basis case: with bases spanning every free degree of freedom and every
entry sampled, the GPU's reduced step equals the full-order step of the same
library and of the oracle.  Trained case: POD bases of the oracle's own
snapshots of a blast run, over-sampled DEIM rows chosen by the oracle; the GPU
reduced step (restricted force on the sampled elements, lifting at their rows,
least-squares projection) against the oracle's full-order-lifted reference,
step by step and under the step control.  The library's own DEIM selection is
compared with the oracle's on a problem without mirror symmetry (no near-tied
rows).  End to end: GPU snapshots, GPU POD and GPU ROM against the oracle's
pipeline, compared through the lifted state (independent of basis signs)."""
import numpy as np
import pytest

import oracle as O
from oracle import rom as OR
from paper_2104_11404_gb300 import workloads as W
from tests._pair import gpu_for, oracle_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sedov(n, **over):
    c = dict(dim=2, n=(n[0], n[1], 1), order=2, problem=W.SEDOV, gamma=1.4, lo=(0.0, 0.0, 0.0),
             hi=(1.0, 1.0, 1.0), visc=1, blast_energy=0.25)
    c.update(over)
    return c


def _rom(g, Pv, Pe, Px, v0, e0, x0, pF, pG):
    from paper_2104_11404_gb300.rom import Rom
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return Rom(g, t(Pv.T), t(Pe.T), t(Px.T), t(v0), t(e0), t(x0), len(pF), len(pG),
               samples_f=pF, samples_g=pG)


def _host(t):
    return t.detach().cpu().numpy()


def test_full_basis_rom_is_the_full_order_step():
    cfg = _sedov((3, 3))
    o = oracle_for(cfg)
    v0, e0, x0 = o.init_state()
    free = np.where(~o.essential_mask())[0]
    Iv = np.eye(o.nv)[:, free]
    Ie = np.eye(o.ne)
    pF, pG = free.copy(), np.arange(o.ne)
    R = OR.RomOracle(o, Iv, Ie, Iv.copy(), v0, e0, x0, pF, pG)
    g = gpu_for(cfg, "fp64")
    r = _rom(g, Iv, Ie, Iv, v0, e0, x0, pF, pG)
    assert r.info.n_elems == o.nelem
    f = gpu_for(cfg, "fp64")
    f.init_state()
    vh, eh, xh = np.zeros(len(free)), np.zeros(o.ne), np.zeros(len(free))
    for dt in (2e-3, 3e-3):
        tau_g = r.step_fixed(dt)
        vh, eh, xh, tau_o = R.step(dt, vh, eh, xh)
        tau_f = f.step_fixed(dt)
        assert abs(tau_g - tau_o) <= 1e-12 * tau_o and abs(tau_g - tau_f) <= 1e-12 * tau_f
        lv, le, lx = (_host(a) for a in r.lift())
        fv, fe, fx, _, _ = f.get_state()
        ov, oe, ox = R.lift(vh, eh, xh)
        for a, b, c in ((lv, _host(fv), ov), (le, _host(fe), oe), (lx, _host(fx), ox)):
            scale = max(np.abs(c).max(), 1e-300)
            assert np.abs(a - c).max() <= 1e-11 * scale
            assert np.abs(a - b).max() <= 1e-11 * scale
    r.close()


def _trained(cfg, t_train, eps=0.9999, over=2):
    """Bases and samples from the oracle's own snapshots of a run."""
    o = oracle_for(cfg)
    v0, e0, x0 = o.init_state()
    v, e, x = v0.copy(), e0.copy(), x0.copy()
    _, Sv, Se, Sx, st = o.run_snapshots(t_train, v, e, x, cap=4000)
    assert st == O.OK
    bases = []
    for S, off in ((Sv, v0), (Se, e0), (Sx, x0)):
        U, sg, k, s2 = O.pod(S, off, eps)
        assert s2 == O.OK and k >= 1
        bases.append(U[:k].T.copy())
    Pv, Pe, Px = bases
    PF, PG = OR.sns_bases(o, Pv, Pe)
    pF = OR.deim(PF, min(over * Pv.shape[1], o.nv))
    pG = OR.deim(PG, min(over * Pe.shape[1], o.ne))
    return o, (v0, e0, x0), (Pv, Pe, Px), pF, pG


def test_trained_rom_matches_oracle_step_by_step_and_under_control():
    cfg = _sedov((8, 8))
    o, (v0, e0, x0), (Pv, Pe, Px), pF, pG = _trained(cfg, 0.1)
    R = OR.RomOracle(o, Pv, Pe, Px, v0, e0, x0, pF, pG)
    g = gpu_for(cfg, "fp64")
    r = _rom(g, Pv, Pe, Px, v0, e0, x0, pF, pG)
    _, sf, sg, els = (r.info, r.samples_f, r.samples_g, r.elements)
    assert np.array_equal(sf, pF) and np.array_equal(sg, pG)
    assert np.array_equal(els, R.els)
    nb = (Pv.shape[1], Pe.shape[1], Px.shape[1])
    vh, eh, xh = (np.zeros(n) for n in nb)
    for dt in (1e-3, 1.5e-3, 2e-3):
        tau_g = r.step_fixed(dt)
        vh, eh, xh, tau_o = R.step(dt, vh, eh, xh)
        assert abs(tau_g - tau_o) <= 1e-11 * tau_o
        gv, ge, gx, _, _ = r.get_state()
        for a, b in ((vh, gv), (eh, ge), (xh, gx)):
            assert np.abs(_host(b) - a).max() <= 1e-10 * max(np.abs(a).max(), 1e-300)
    # the step control from the initial state
    r.set_state(np.zeros(nb[0]), np.zeros(nb[1]), np.zeros(nb[2]))
    st = r.run_to(0.1)
    ovh, oeh, oxh, t, dt, steps, rejects, log = R.run(0.1, *(np.zeros(n) for n in nb))
    assert st["steps"] == steps and st["rejects"] == rejects and st["t"] == 0.1
    gv, ge, gx, _, _ = r.get_state()
    for a, b in ((ovh, gv), (oeh, ge), (oxh, gx)):
        assert np.abs(_host(b) - a).max() <= 1e-9 * max(np.abs(a).max(), 1e-300)
    # the reduced model reproduces its own training run closely
    fv, fe, fx = o.init_state()
    o.run(0.1, fv, fe, fx)
    lv, le, lx = (_host(a) for a in r.lift())
    assert np.linalg.norm(lv - fv) <= 1e-2 * np.linalg.norm(fv)
    assert np.linalg.norm(lx - fx) <= 1e-3 * np.linalg.norm(fx)
    r.close()


def test_library_deim_selection_matches_oracle():
    cfg = dict(W.CONFIGS["triple3d_28"], dim=2, n=(14, 6, 1))
    o, (v0, e0, x0), (Pv, Pe, Px), pF, pG = _trained(cfg, 0.3)
    from paper_2104_11404_gb300.rom import Rom
    g = gpu_for(cfg, "fp64")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    r = Rom(g, t(Pv.T), t(Pe.T), t(Px.T), t(v0), t(e0), t(x0), len(pF), len(pG))
    assert np.array_equal(r.samples_f, pF)
    assert np.array_equal(r.samples_g, pG)
    r.close()


def test_gpu_offline_and_online_pipeline_matches_oracle():
    """GPU snapshots (batched run) -> GPU POD -> GPU ROM, against the same
    pipeline in the oracle, compared through the lifted final state."""
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300.batch import Batch
    cfg = _sedov((8, 8))
    t_train = 0.1
    o, (v0, e0, x0), (Pv, Pe, Px), pF, pG = _trained(cfg, t_train)
    R = OR.RomOracle(o, Pv, Pe, Px, v0, e0, x0, pF, pG)
    ovh, oeh, oxh, *_ = R.run(t_train, *(np.zeros(P.shape[1]) for P in (Pv, Pe, Px)))
    ov, oe, ox = R.lift(ovh, oeh, oxh)
    b = Batch([cfg], precision="fp64")
    b.init_state()
    gv0, ge0, gx0 = (a.clone() for a in b.get_state())
    Sv, Se, Sx = b.snapshots([0], 4000)
    b.run_to(t_train)
    (_, cnt, V, E, X), = b.snapshot_views(Sv, Se, Sx)
    gb = []
    for cols, off in ((V, gv0), (E, ge0), (X, gx0)):
        n, m = cols.shape
        U = torch.zeros(n * m, dtype=torch.float64, device="cuda")
        sig = torch.zeros(n, dtype=torch.float64, device="cuda")
        work = torch.zeros(m * n + 2 * n + 16, dtype=torch.float64, device="cuda")
        k, _ = lagh.lh_pod(cols.contiguous(), m, n, off, 0.9999, U, sig, work,
                           torch.cuda.current_stream().cuda_stream)
        gb.append(U.view(n, m)[:k].contiguous())
    b.close()
    assert [B.shape[0] for B in gb] == [Pv.shape[1], Pe.shape[1], Px.shape[1]]
    from paper_2104_11404_gb300.rom import Rom
    g = gpu_for(cfg, "fp64")
    # the oracle's sample rows (the blast is mirror-symmetric: rows tie in
    # pairs, and which of a pair is taken depends on rounding)
    r = Rom(g, gb[0], gb[1], gb[2], gv0, ge0, gx0, len(pF), len(pG), samples_f=pF, samples_g=pG)
    r.run_to(t_train)
    lv, le, lx = (_host(a) for a in r.lift())
    assert np.linalg.norm(lv - ov) <= 1e-6 * np.linalg.norm(ov)
    assert np.linalg.norm(le - oe) <= 1e-6 * np.linalg.norm(oe)
    assert np.linalg.norm(lx - ox) <= 1e-8 * np.linalg.norm(ox)
    r.close()


def test_mixed_rom_follows_the_fp64_reduced_model():
    """The hyper-reduced step on a mixed context (FP32 stress and F_K of the
    sampled elements, error-free F.1 / F^T w sums, FP64 reduced state): step
    by step within FP32 accuracy of the oracle's FP64 reduced step, and under
    the step control to t = 0.1 within 1e-4 of the oracle's reduced run."""
    cfg = _sedov((8, 8))
    o, (v0, e0, x0), (Pv, Pe, Px), pF, pG = _trained(cfg, 0.1)
    R = OR.RomOracle(o, Pv, Pe, Px, v0, e0, x0, pF, pG)
    g = gpu_for(cfg, "mixed")
    r = _rom(g, Pv, Pe, Px, v0, e0, x0, pF, pG)
    nb = (Pv.shape[1], Pe.shape[1], Px.shape[1])
    vh, eh, xh = (np.zeros(n) for n in nb)
    for dt in (1e-3, 1.5e-3, 2e-3):
        tau_g = r.step_fixed(dt)
        vh, eh, xh, tau_o = R.step(dt, vh, eh, xh)
        assert abs(tau_g - tau_o) <= 1e-5 * tau_o
        gv, ge, gx, _, _ = r.get_state()
        for a, b in ((vh, gv), (eh, ge), (xh, gx)):
            assert np.abs(_host(b) - a).max() <= 1e-5 * max(np.abs(a).max(), 1e-300)
    r.set_state(np.zeros(nb[0]), np.zeros(nb[1]), np.zeros(nb[2]))
    st = r.run_to(0.1)
    ovh, oeh, oxh, t, dt, steps, rejects, log = R.run(0.1, *(np.zeros(n) for n in nb))
    assert st["t"] == 0.1 and abs(st["steps"] - steps) <= 2
    ov, oe, ox = R.lift(ovh, oeh, oxh)
    lv, le, lx = (_host(a) for a in r.lift())
    assert np.linalg.norm(lv - ov) <= 1e-4 * np.linalg.norm(ov)
    assert np.linalg.norm(le - oe) <= 1e-4 * np.linalg.norm(oe)
    assert np.linalg.norm(lx - ox) <= 1e-6 * np.linalg.norm(ox)
    r.close()
