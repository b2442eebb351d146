"""Host logic of bench.py on CPU: the replica (multi-GPU) timing aggregation
under torch.distributed with the gloo backend at world size 2, and the
reference arm's rank handling."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    # rank r took 100 (r + 1) ms for its 5 instances: the job takes the slowest rank's time
    value, total = bench.job_throughput(100.0 * (rank + 1), 5, dist, "cpu")
    q.put((rank, value, total))
    dist.destroy_process_group()


def test_replica_throughput_is_max_over_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, value, total in got:
        assert total == pytest.approx(200.0)
        assert value == pytest.approx(2 * 5 / 0.2)     # 10 instances in 0.2 s


def test_single_process_throughput():
    sys.path.insert(0, ROOT)
    import bench
    value, total = bench.job_throughput(250.0, 5)
    assert total == 250.0 and value == pytest.approx(20.0)


def test_reference_arm_non_zero_rank_does_no_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    ns = type("A", (), {"interface_solves": 18, "workload": "star128", "warmup": 1, "steps": 1,
                        "gpus": 2})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main_reference(ns)
    assert buf.getvalue() == ""


def test_host_cpu_description_is_json():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.host_cpu()
    assert h["logical_cpus"] == os.cpu_count() and h["machine"]
    json.dumps(h)


def test_reference_arm_scales_by_the_workload_interface_solves(monkeypatch):
    """Without --interface-solves the reference arm scales one oracle matvec by
    the workload's own count (star128: 59 GMRES iterations + 2 solves)."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(bench, "run_oracle_subprocess",
                        lambda workload, reps, per_solve: {"times": [2.0] * reps})
    ns = type("A", (), {"interface_solves": None, "workload": "star128", "warmup": 1, "steps": 2,
                        "gpus": 1})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main_reference(ns)
    line = json.loads(buf.getvalue())
    assert bench.INTERFACE_SOLVES["star128"] == 61
    assert line["value"] == pytest.approx(1.0 / (2.0 * 61), rel=1e-4)
    assert "61 interface solves" in line["cpu_baseline"]["sample"]
    ns.workload = "star64"
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main_reference(ns)
    assert "unavailable" in json.loads(buf.getvalue())
