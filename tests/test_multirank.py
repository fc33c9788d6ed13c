"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups.

bench.py runs one replica per GPU (no collective on the data path). Its only
cross-rank operations are the max of the timed region and the sums of the
processed units, and under torchrun the reference arm runs on rank 0 alone.
Both are host logic, tested here with gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r processed 100 (r + 1) units in 1 + r ms
    units = bench.rank_reduce(100.0 * (rank + 1), "sum", world, "cpu")
    ms = bench.rank_reduce(1.0 + rank, "max", world, "cpu")
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()
    out.put((rank, units, ms))


def test_rank_reduce_sums_units_and_takes_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the whole-job sums and the max time: 300 units in 2 ms
    assert res == [(0, 300.0, 2.0), (1, 300.0, 2.0)]


def test_rank_reduce_is_the_identity_at_world_size_one():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_reduce(7.5, "max", 1, "cpu") == 7.5
    assert bench.rank_reduce(7.5, "sum", 1, "cpu") == 7.5


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
