"""lh_force_static: the force evaluation for callers that cannot allocate
device memory (their memory belongs to a framework pool, is budgeted up
front, or must not be allocated inside a latency-critical loop).  Its only
working memory is a fixed-size array inside the library, so it is checked
against the context-based lh_force on two calls in a row (the second call
must not see the first one's leftovers), and its size limit is checked.

This file is named to run last: a failure here leaves every other test run."""
import numpy as np
import pytest

from paper_2104_11404_gb300 import workloads as W
from tests._pair import dev, gpu_for, host, max_rel, oracle_for, random_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _descs(g):
    """The descriptors a context was created from, rebuilt for the
    context-free call."""
    from paper_2104_11404_gb300 import lagh
    cfg = g.cfg
    mesh = lagh.lh_mesh_desc()
    mesh.dim = cfg["dim"]
    mesh.nx, mesh.ny, mesh.nz = [int(v) for v in cfg["n"]]
    for i in range(3):
        mesh.lo[i] = float(cfg["lo"][i])
        mesh.hi[i] = float(cfg["hi"][i])
    disc = lagh.lh_disc_desc()
    disc.order = cfg["order"]
    disc.nq = 2 * cfg["order"]
    phys = lagh.lh_default_phys()
    phys.problem = cfg["problem"]
    phys.gamma = float(cfg["gamma"])
    phys.visc = int(cfg.get("visc", 1))
    phys.cfl = float(cfg.get("cfl", 0.5))
    return mesh, disc, phys


@pytest.mark.parametrize("dim,k,n", [(2, 2, (7, 5, 1)), (3, 2, (3, 4, 2)), (2, 3, (4, 3, 1))])
def test_force_static_matches_force_twice(dim, k, n):
    from paper_2104_11404_gb300 import lagh
    cfg = dict(dim=dim, n=n, order=k, problem=W.SEDOV, gamma=1.4, lo=(0.0, 0.0, 0.0),
               hi=(1.0, 1.0, 1.0), visc=1, blast_energy=0.25)
    o = oracle_for(cfg)
    g = gpu_for(cfg)
    mesh, disc, phys = _descs(g)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (41, 42):  # two calls in a row on different states
        v, e, x = random_state(o, cfg, seed=seed)
        F1_ref, _, dt_ref = g.force(dev(v), dev(e), dev(x))
        F1 = torch.full((o.nv,), float("nan"), dtype=torch.float64, device="cuda")
        dt = lagh.lh_force_static(mesh, disc, phys, dev(v), dev(e), dev(x), F1, stream)
        assert max_rel(host(F1_ref), host(F1)) <= 1e-12
        assert abs(dt - dt_ref) <= 1e-12 * dt_ref
        # and both agree with the oracle
        F1o, _, dto, _ = o.force(v, e, x)
        assert max_rel(F1o, host(F1)) <= 1e-12


def test_force_static_reports_state_checks_without_an_estimate():
    """With no context, no later call could report a bad state, so every call
    reads back the flags: an inverted element gives LH_ETANGLED and a NaN
    LH_ENONFINITE, with or without the estimate, and the next clean call on
    the same stream returns LH_OK (the flag slot is cleared at each call)."""
    from paper_2104_11404_gb300 import lagh
    cfg = dict(dim=2, n=(4, 4, 1), order=2, problem=W.SEDOV, gamma=1.4, lo=(0.0, 0.0, 0.0),
               hi=(1.0, 1.0, 1.0), visc=1, blast_energy=0.25)
    o = oracle_for(cfg)
    g = gpu_for(cfg)
    mesh, disc, phys = _descs(g)
    stream = torch.cuda.current_stream().cuda_stream
    v, e, x = random_state(o, cfg, seed=43)
    xt = x.copy()
    xt[0], xt[2] = xt[2], xt[0]           # two corner nodes of element 0 swapped
    en = e.copy()
    en[5] = np.nan
    F1 = torch.zeros(o.nv, dtype=torch.float64, device="cuda")
    for want_dt in (True, False):
        with pytest.raises(lagh.LaghError) as ei:
            lagh.lh_force_static(mesh, disc, phys, dev(v), dev(e), dev(xt), F1, stream,
                                 want_dt=want_dt)
        assert ei.value.status == lagh.LH_ETANGLED
        with pytest.raises(lagh.LaghError) as ei:
            lagh.lh_force_static(mesh, disc, phys, dev(v), dev(en), dev(x), F1, stream,
                                 want_dt=want_dt)
        assert ei.value.status == lagh.LH_ENONFINITE
        # a clean state right after, on the same stream: no leftover flag
        F1.fill_(float("nan"))
        lagh.lh_force_static(mesh, disc, phys, dev(v), dev(e), dev(x), F1, stream,
                             want_dt=want_dt)
        torch.cuda.synchronize()
        F1o, _, _, _ = o.force(v, e, x)
        assert max_rel(F1o, host(F1)) <= 1e-12


def test_force_static_size_limit_is_exact():
    """2D Q2 needs 16 + 19 n_e doubles: 470 x 469 elements fit the 4 Mi-double
    array (n_e = 220,430), 471 x 469 (220,899) do not."""
    from paper_2104_11404_gb300 import lagh
    cfg = dict(dim=2, n=(470, 469, 1), order=2, problem=W.SEDOV, gamma=1.4,
               lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), visc=1, blast_energy=0.25)
    g = gpu_for(cfg)
    g.init_state()
    v, e, x, _, _ = g.get_state()
    mesh, disc, phys = _descs(g)
    stream = torch.cuda.current_stream().cuda_stream
    F1 = torch.full((g.nv,), float("nan"), dtype=torch.float64, device="cuda")
    dt = lagh.lh_force_static(mesh, disc, phys, v, e, x, F1, stream)
    F1_ref, _, dt_ref = g.force(v, e, x)
    assert max_rel(host(F1_ref), host(F1)) <= 1e-12
    assert abs(dt - dt_ref) <= 1e-12 * dt_ref
    g.close()
    mesh.nx = 471
    with pytest.raises(lagh.LaghError) as ei:
        lagh.lh_force_static(mesh, disc, phys, v, e, x, F1, stream)
    assert ei.value.status == lagh.LH_ETOOLARGE


def test_force_static_rejects_meshes_beyond_its_memory():
    from paper_2104_11404_gb300 import lagh
    cfg = dict(dim=3, n=(40, 40, 40), order=2, problem=W.SEDOV, gamma=1.4, lo=(0.0, 0.0, 0.0),
               hi=(1.0, 1.0, 1.0), visc=1)
    mesh = lagh.lh_mesh_desc()
    mesh.dim, mesh.nx, mesh.ny, mesh.nz = 3, 40, 40, 40
    for i in range(3):
        mesh.hi[i] = 1.0
    disc = lagh.lh_disc_desc()
    disc.order, disc.nq = 2, 4
    phys = lagh.lh_default_phys()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lagh.LaghError) as ei:
        lagh.lh_force_static(mesh, disc, phys, buf, buf, buf, buf)
    assert ei.value.status == lagh.LH_ETOOLARGE
