"""Batched form against the oracle, instance by instance.

Each instance of a batch follows the step of a single problem; the oracle
advances the same instance alone.  Per-step parity uses the same random
states and step sizes on both sides; full runs compare the step control's
decisions and the final fields; the restricted force compares element rows
with the oracle's dense element matrices."""
import numpy as np
import pytest

from paper_2104_11404_gb300 import workloads as W
from tests._pair import dev, gpu_for, host, max_rel, oracle_for, random_state, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sedov(n, gamma=1.4, e0=0.25, **over):
    c = dict(dim=2, n=tuple(n) + (1,) * (3 - len(n)), order=2, problem=W.SEDOV, gamma=gamma,
             lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1, blast_energy=e0, t_final=0.8)
    c.update(over)
    return c


def _batch(cfgs, precision="fp64", **kw):
    from paper_2104_11404_gb300.batch import Batch
    return Batch(cfgs, precision=precision, **kw)


def _pack(parts):
    return np.concatenate(parts) if parts else np.zeros(0)


def _random_batch_state(cfgs, seed):
    os_, vs, es, xs = [], [], [], []
    for i, c in enumerate(cfgs):
        o = oracle_for(c)
        v, e, x = random_state(o, c, seed=seed + i)
        os_.append(o)
        vs.append(v)
        es.append(e)
        xs.append(x)
    return os_, vs, es, xs


MIXED_SET = [_sedov((6, 5), 1.4, 0.25), _sedov((4, 4), 1.6, 0.7), _sedov((7, 3), 1.33, 0.1)]
FP64_SET = MIXED_SET + [dict(W.scaled("tg2d_64", n=(5, 4)))]


@pytest.mark.parametrize("precision,tol,cfgs", [("fp64", 1e-12, FP64_SET),
                                                ("mixed", 1e-5, MIXED_SET)])
def test_batch_step_fixed_matches_oracle_per_instance(precision, tol, cfgs):
    os_, vs, es, xs = _random_batch_state(cfgs, seed=70)
    b = _batch(cfgs, precision)
    b.set_state(dev(_pack(vs)), dev(_pack(es)), dev(_pack(xs)))
    rng = np.random.default_rng(5)
    for rep in range(2):  # two steps in a row, different step sizes
        dts = np.array([1e-3 * (1.0 + rng.uniform()) for _ in cfgs])
        st = b.step_fixed(dts)
        assert st["steps"] == len(cfgs)
        for i, o in enumerate(os_):
            _, _, s = o.step(float(dts[i]), vs[i], es[i], xs[i])
            assert s == 0
        vg, eg, xg = b.get_state()
        for i in range(len(cfgs)):
            gv, ge, gx = (host(t) for t in b.instance(i, vg, eg, xg))
            assert max_rel(vs[i], gv) <= tol, (precision, i, rep)
            assert max_rel(es[i], ge) <= tol, (precision, i, rep)
            assert max_rel(xs[i], gx) <= tol * 1e-2, (precision, i, rep)
    q = b.query()  # counters of the last run (one step)
    assert np.all(q["steps"] == 1) and np.all(q["status"] == 0)
    assert np.all(q["cg_iters"] >= 2)


def test_batch_sedov_free_running_matches_oracle_fp64():
    """Every instance runs its own step control to t = 0.3."""
    cfgs = [_sedov((6, 6), 1.4, 0.25), _sedov((8, 8), 1.55, 0.6), _sedov((5, 7), 1.35, 0.15)]
    t_final = 0.3
    b = _batch(cfgs, "fp64")
    b.init_state()
    E0 = b.total_energy()
    st = b.run_to(t_final)
    q = b.query()
    vg, eg, xg = b.get_state()
    E1 = b.total_energy()
    assert st["instances_done"] == len(cfgs)
    for i, c in enumerate(cfgs):
        o = oracle_for(c)
        v, e, x = o.init_state()
        Eo = o.total_energy(v, e)
        assert abs(E0[i] - Eo) <= 1e-12 * Eo
        stats, log, s = o.run(t_final, v, e, x)
        assert s == 0
        assert q["t"][i] == t_final
        assert q["steps"][i] == stats["steps"] and q["rejects"][i] == stats["rejects"]
        gv, ge, gx = (host(t) for t in b.instance(i, vg, eg, xg))
        assert rel_l2(v, gv) <= 1e-8 and rel_l2(e, ge) <= 1e-8 and rel_l2(x, gx) <= 1e-8
        assert abs(E1[i] - E0[i]) <= 1e-12 * E0[i]
    # one CG iteration per solve: the preconditioner is the exact inverse
    assert np.all(q["cg_iters"] == 2 * (q["steps"] + q["rejects"]))
    assert st["dof_updates"] == int(np.sum(b.dofs() * q["steps"]))


def test_batch_sedov_mixed_energy_and_accuracy():
    cfgs = [_sedov((8, 8), 1.4, 0.25), _sedov((6, 6), 1.6, 0.9)]
    t_final = 0.3
    b = _batch(cfgs, "mixed")
    b.init_state()
    E0 = b.total_energy()
    b.run_to(t_final)
    E1 = b.total_energy()
    vg, eg, xg = b.get_state()
    for i, c in enumerate(cfgs):
        assert abs(E1[i] - E0[i]) <= 1e-10 * E0[i]
        o = oracle_for(c)
        v, e, x = o.init_state()
        o.run(t_final, v, e, x)
        gv, ge, gx = (host(t) for t in b.instance(i, vg, eg, xg))
        assert rel_l2(v, gv) <= 1e-4 and rel_l2(e, ge) <= 1e-4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_batch_force_sampled_rows(precision, tol):
    from tests import _fem_ref as R
    cfgs = [_sedov((6, 5)), _sedov((9, 4), 1.5), _sedov((5, 5), 1.62)]
    os_, vs, es, xs = _random_batch_state(cfgs, seed=90)
    ws = [random_state(o, c, seed=190 + i)[0] for i, (o, c) in enumerate(zip(os_, cfgs))]
    b = _batch(cfgs, precision)
    lists = [W.element_sample(o.nelem, frac=0.3, stream=i) for i, o in enumerate(os_)]
    lists[2] = np.zeros(0, dtype=np.int32)  # an instance with no sampled element
    F1, FTv, off, dts = b.force_sampled(lists, dev(_pack(vs)), dev(_pack(es)), dev(_pack(xs)),
                                        vtest=dev(_pack(ws)))
    F1, FTv = host(F1), host(FTv)
    for i, (o, c) in enumerate(zip(os_, cfgs)):
        mesh = R.CartesianMesh(2, c["n"][:2], 2)
        rows = F1[off[i] * 2 * o.nd1: off[i + 1] * 2 * o.nd1].reshape(-1, 2 * o.nd1)
        frows = FTv[off[i] * o.nd2: off[i + 1] * o.nd2].reshape(-1, o.nd2)
        for s, el in enumerate(lists[i]):
            FK = o.element_force_matrix(int(el), vs[i], es[i], xs[i])
            cn = mesh.conn(int(el))
            wl = np.concatenate([ws[i][cc * o.nnodes + cn] for cc in range(2)])
            assert max_rel(FK.sum(axis=1), rows[s]) <= tol
            assert max_rel(FK.T @ wl, frows[s]) <= tol
        if len(lists[i]):
            g = gpu_for(c, precision=precision)
            _, _, dt1 = g.force_sampled(dev(lists[i]), dev(vs[i]), dev(es[i]), dev(xs[i]))
            assert abs(dts[i] - dt1) <= 1e-12 * dt1
        else:
            assert dts[i] == np.inf


def test_batch_launch_shapes_agree_and_autotune_keeps_state():
    cfgs = [_sedov((6, 6), 1.4, 0.25), _sedov((10, 4), 1.5, 0.5), _sedov((3, 3), 1.45, 0.3)]
    os_, vs, es, xs = _random_batch_state(cfgs, seed=11)
    dts = np.array([1e-3, 1.5e-3, 0.7e-3])
    ref = None
    shapes = [(t, sl, 1) for t in (256, 512, 1024) for sl in (2, 1, 0)]
    shapes += [(t, 2, 2) for t in (256, 512, 1024)]  # two quadrature points per thread
    for threads, sl, qpt in shapes:
            b = _batch(cfgs, "mixed", tuning=dict(threads=threads, ctas_per_sm=1, smem_lines=sl,
                                                  qpt=qpt))
            assert b.tuning()["threads"] == threads and b.tuning()["qpt"] == qpt
            b.set_state(dev(_pack(vs)), dev(_pack(es)), dev(_pack(xs)))
            b.step_fixed(dts)
            out = [host(t) for t in b.get_state()]
            if ref is None:
                ref = out
            else:
                for a, c in zip(ref, out):
                    assert max_rel(a, c) <= 1e-12
            b.close()
    b = _batch(cfgs, "mixed")
    b.set_state(dev(_pack(vs)), dev(_pack(es)), dev(_pack(xs)))
    before = [host(t) for t in b.get_state()]
    q0 = b.query()
    chosen = b.autotune(reps=1)
    assert chosen["threads"] in (256, 512, 1024) and chosen["ctas_per_sm"] >= 1
    assert chosen["qpt"] in (1, 2)
    after = [host(t) for t in b.get_state()]
    for a, c in zip(before, after):
        assert np.array_equal(a, c)
    q1 = b.query()
    assert np.array_equal(q0["t"], q1["t"]) and np.array_equal(q0["cg_iters"], q1["cg_iters"])
    b.step_fixed(dts)
    out = [host(t) for t in b.get_state()]
    for a, c in zip(ref, out):
        assert max_rel(a, c) <= 1e-12


def test_batch_more_instances_than_ctas():
    """Instances outnumber the persistent CTAs: every CTA takes several."""
    rng = np.random.default_rng(3)
    cfgs = [_sedov((int(rng.integers(2, 5)), int(rng.integers(2, 5))), 1.3 + 0.3 * rng.uniform(),
                   0.1 + 0.9 * rng.uniform()) for _ in range(400)]
    b = _batch(cfgs, "fp64", tuning=dict(threads=256, ctas_per_sm=1, smem_lines=1))
    b.init_state()
    st = b.run_to(0.05)
    assert st["instances_done"] == len(cfgs)
    vg, eg, xg = b.get_state()
    q = b.query()
    for i in (0, 137, 399):
        o = oracle_for(cfgs[i])
        v, e, x = o.init_state()
        stats, _, s = o.run(0.05, v, e, x)
        assert q["steps"][i] == stats["steps"]
        gv, ge, gx = (host(t) for t in b.instance(i, vg, eg, xg))
        assert rel_l2(v, gv) <= 1e-8 and rel_l2(e, ge) <= 1e-8


def test_batch_invalid_arguments_and_finished_instances():
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300.hydro import descriptors
    m2, d2, p2 = descriptors(_sedov((4, 4)))
    m3, _, p3 = descriptors(dict(_sedov((2, 2)), dim=3, n=(2, 2, 2)))
    with pytest.raises(lagh.LaghError) as ei:
        lagh.lh_batch_create([m2, m3], d2, [p2, p3], lagh.LH_FP64)
    assert ei.value.status == lagh.LH_EINVAL
    with pytest.raises(lagh.LaghError):
        lagh.lh_batch_create([], d2, [], lagh.LH_FP64)
    b = _batch([_sedov((4, 4)), _sedov((3, 5))])
    b.init_state()
    with pytest.raises(lagh.LaghError) as ei:
        b.step_fixed(np.array([1e-3, 0.0]))
    assert ei.value.status == lagh.LH_EINVAL
    st = b.run_to(0.0)  # already at t_final: nothing to do
    assert st["steps"] == 0 and st["instances_done"] == 2
    st = b.run_to(0.05, max_steps=3)
    q = b.query()
    assert np.all(q["steps"] == 3) and st["steps"] == 6


def test_batch_bench_workload_instances_match_single_contexts():
    """The 512-instance point-blast sweep (mixed) as the benchmark runs it:
    a few attempts of the whole batch after autotuning; one instance of each
    mesh size against a single-problem context and the FP64 oracle, and the
    energy balance of every instance."""
    cfgs = W.batch_instances()
    b = _batch(cfgs, "mixed")
    b.init_state()
    b.autotune(reps=1)
    E0 = b.total_energy()
    steps = 3
    st = b.run_to(0.8, max_steps=steps)
    q = b.query()
    assert np.all(q["status"] == 0) and np.all(q["steps"] == steps)
    E1 = b.total_energy()
    assert np.max(np.abs(E1 - E0) / E0) <= 1e-10
    vg, eg, xg = b.get_state()
    seen = set()
    for i, c in enumerate(cfgs):
        if c["n"][0] in seen:
            continue
        seen.add(c["n"][0])
        g = gpu_for(c, precision="mixed")
        g.init_state()
        g.run_to(0.8, max_steps=steps)
        v1, e1, x1, t1, _ = g.get_state()
        gv, ge, gx = b.instance(i, vg, eg, xg)
        assert abs(q["t"][i] - t1) <= 1e-12 * t1
        assert rel_l2(host(v1), host(gv)) <= 1e-6 and rel_l2(host(e1), host(ge)) <= 1e-6
        o = oracle_for(c)
        v, e, x = o.init_state()
        o.run(0.8, v, e, x, max_steps=steps)
        assert rel_l2(v, host(gv)) <= 1e-4 and rel_l2(e, host(ge)) <= 1e-4
    assert len(seen) == len(W.BATCH_SIZES)


@pytest.mark.parametrize("dim,k,sizes", [(2, 1, [(6, 5), (4, 7)]), (2, 3, [(3, 4), (5, 3)]),
                                          (3, 1, [(3, 3, 2), (2, 4, 3)]),
                                          (3, 2, [(2, 3, 2), (3, 2, 2)])])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_batch_other_orders_and_3d_per_step(dim, k, sizes, precision, tol):
    """Other orders and 3D instances (3D node lines are solved in device
    memory, the mass apply in element tiles) against the oracle, two steps."""
    cfgs = []
    for i, n in enumerate(sizes):
        cfgs.append(dict(dim=dim, n=tuple(n) + (1,) * (3 - len(n)), order=k, problem=W.SEDOV,
                         gamma=1.4 + 0.1 * i, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1,
                         blast_energy=0.25 + 0.2 * i, t_final=0.8))
    os_, vs, es, xs = _random_batch_state(cfgs, seed=300 + 10 * dim + k)
    b = _batch(cfgs, precision)
    b.set_state(dev(_pack(vs)), dev(_pack(es)), dev(_pack(xs)))
    for rep in range(2):
        dts = np.array([8e-4 * (1 + 0.3 * i + 0.1 * rep) for i in range(len(cfgs))])
        b.step_fixed(dts)
        for i, o in enumerate(os_):
            _, _, s = o.step(float(dts[i]), vs[i], es[i], xs[i])
            assert s == 0
        vg, eg, xg = b.get_state()
        for i in range(len(cfgs)):
            gv, ge, gx = (host(t) for t in b.instance(i, vg, eg, xg))
            assert max_rel(vs[i], gv) <= tol and max_rel(es[i], ge) <= tol, (i, rep)
    q = b.query()
    assert np.all(q["status"] == 0)
