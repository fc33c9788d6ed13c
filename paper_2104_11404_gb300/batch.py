"""Convenience wrapper of a library batch (many independent instances) for
Python users: descriptors from configuration dicts, packed torch tensors
through the C ABI.  All computation happens in liblagh.so."""
import numpy as np
import torch

from . import lagh
from .hydro import descriptors, precision_id


class Batch:
    def __init__(self, cfgs, precision="mixed", stream=None, cg_rtol=None, cg_maxit=None,
                 tuning=None, phys_overrides=None):
        L = lagh
        self.precision = precision_id(precision)
        if tuning is not None:
            unknown = set(tuning) - {"threads", "ctas_per_sm", "smem_lines", "qpt"}
            if unknown:
                raise KeyError("unknown tuning keys %s" % sorted(unknown))
        self.cfgs = [dict(c) for c in cfgs]
        meshes, physs = [], []
        disc = None
        for c in self.cfgs:
            m, d, p = descriptors(c, cg_rtol, cg_maxit, phys_overrides)
            meshes.append(m)
            physs.append(p)
            disc = disc or d
        self.n = len(self.cfgs)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        tun = None
        if tuning is not None:
            tun = L.lh_batch_tuning()
            tun.threads = int(tuning.get("threads", 0))
            tun.ctas_per_sm = int(tuning.get("ctas_per_sm", 0))
            tun.smem_lines = int(tuning.get("smem_lines", 1))
            tun.qpt = int(tuning.get("qpt", 1))
        self.b = L.lh_batch_create(meshes, disc, physs, self.precision, self.stream.cuda_stream,
                                   tun)
        off_v, off_e, info = L.lh_batch_layout(self.b, self.n)
        self.off_v, self.off_e, self.info = np.array(off_v), np.array(off_e), info
        self.nv, self.ne = int(off_v[-1]), int(off_e[-1])
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "b", None):
            lagh.lh_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dofs(self):
        """2 N_V + N_E of every instance."""
        return np.array([2 * i.nv + i.ne for i in self.info], dtype=np.int64)

    def init_state(self):
        lagh.lh_batch_init_state(self.b)

    def set_state(self, v, e, x, t=None, dt=None):
        t = None if t is None else np.ascontiguousarray(t, dtype=np.float64)
        dt = None if dt is None else np.ascontiguousarray(dt, dtype=np.float64)
        lagh.lh_batch_set_state(self.b, v, e, x, t, dt)

    def get_state(self):
        v = torch.zeros(self.nv, dtype=torch.float64, device=self.dev)
        x = torch.zeros(self.nv, dtype=torch.float64, device=self.dev)
        e = torch.zeros(self.ne, dtype=torch.float64, device=self.dev)
        lagh.lh_batch_get_state(self.b, v, e, x)
        return v, e, x

    def instance(self, i, v, e, x):
        """Views of instance i in packed arrays."""
        a, b = int(self.off_v[i]), int(self.off_v[i + 1])
        c, d = int(self.off_e[i]), int(self.off_e[i + 1])
        return v[a:b], e[c:d], x[a:b]

    def query(self):
        n = self.n
        out = dict(t=np.zeros(n), dt=np.zeros(n), steps=np.zeros(n, np.int64),
                   rejects=np.zeros(n, np.int64), cg_iters=np.zeros(n, np.int64),
                   status=np.zeros(n, np.int32))
        lagh.lh_batch_query(self.b, out["t"], out["dt"], out["steps"], out["rejects"],
                            out["cg_iters"], out["status"])
        return out

    def run_to(self, t_final, max_steps=2 ** 62):
        return lagh.lh_batch_run_to(self.b, t_final, max_steps)

    def step_fixed(self, dt):
        return lagh.lh_batch_step_fixed(self.b, np.ascontiguousarray(dt, dtype=np.float64))

    def total_energy(self):
        out = np.zeros(self.n)
        lagh.lh_batch_total_energy(self.b, out)
        return out

    def force_sampled(self, lists, v=None, e=None, x=None, vtest=None):
        """lists: one int32 array of element ids per instance.  Returns the
        packed element rows of F.1 (and F^T vtest), the offsets and the
        per-instance estimates."""
        counts = np.array([len(l) for l in lists], dtype=np.int64)
        off = np.zeros(self.n + 1, dtype=np.int64)
        off[1:] = np.cumsum(counts)
        ids = np.concatenate([np.asarray(l, dtype=np.int32) for l in lists]) if off[-1] else \
            np.zeros(0, dtype=np.int32)
        d_off = torch.from_numpy(off).to(self.dev)
        d_ids = torch.from_numpy(ids).to(self.dev)
        i0 = self.info[0]
        F1 = torch.zeros(int(off[-1]) * i0.dim * i0.ndof_h1, dtype=torch.float64, device=self.dev)
        FTv = (torch.zeros(int(off[-1]) * i0.ndof_l2, dtype=torch.float64, device=self.dev)
               if vtest is not None else None)
        dt = np.zeros(self.n)
        lagh.lh_batch_force_sampled(self.b, d_off, d_ids, F1, v, e, x, vtest, FTv, dt)
        return F1, FTv, off, dt

    def snapshots(self, ids, cap):
        """Arms snapshot capture (lh_batch_snapshots) for the instances `ids`
        with room for `cap` columns each; returns the packed device matrices
        (Sv, Se, Sx) and per selected instance its (row count v, row count
        e, column offset v, column offset e)."""
        ids = sorted(int(i) for i in ids)
        nv = [self.info[i].nv for i in ids]
        ne = [self.info[i].ne for i in ids]
        Sv = torch.zeros(cap * sum(nv), dtype=torch.float64, device=self.dev)
        Sx = torch.zeros(cap * sum(nv), dtype=torch.float64, device=self.dev)
        Se = torch.zeros(cap * sum(ne), dtype=torch.float64, device=self.dev)
        lagh.lh_batch_snapshots(self.b, ids, cap, Sv, Se, Sx)
        self._snap = (ids, cap, nv, ne)
        return Sv, Se, Sx

    def snapshot_views(self, Sv, Se, Sx):
        """Per selected instance: (id, count, V [cols, N_V], E [cols, N_E], X
        [cols, N_V]) views of the captured columns."""
        ids, cap, nv, ne = self._snap
        cnt = lagh.lh_batch_snapshot_count(self.b, self.n)
        out, ov, oe = [], 0, 0
        for s, i in enumerate(ids):
            c = min(cnt[i], cap)
            V = Sv[ov:ov + cap * nv[s]].view(cap, nv[s])[:c]
            X = Sx[ov:ov + cap * nv[s]].view(cap, nv[s])[:c]
            E = Se[oe:oe + cap * ne[s]].view(cap, ne[s])[:c]
            out.append((i, cnt[i], V, E, X))
            ov += cap * nv[s]
            oe += cap * ne[s]
        return out

    def autotune(self, reps=2):
        t = lagh.lh_batch_autotune(self.b, reps)
        return dict(threads=t.threads, ctas_per_sm=t.ctas_per_sm, smem_lines=t.smem_lines,
                    qpt=t.qpt)

    def tuning(self):
        t = lagh.lh_batch_tuning_get(self.b)
        return dict(threads=t.threads, ctas_per_sm=t.ctas_per_sm, smem_lines=t.smem_lines,
                    qpt=t.qpt)
