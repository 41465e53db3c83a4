"""The multi-process side of the benchmark on the CPU: world size 2 over
gloo.  Every rank is an independent replica (the method exchanges nothing
between cases), the step time is the slowest rank's, and the CPU oracle arm
runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # per-rank device times of one replica; the job time is the maximum
        t = bench.max_over_ranks(dist, 1.0 + 0.5 * rank, "cpu")
        units = 1000 * 3 * 10 * ws          # fluid cells x species x steps x replicas
        out[rank] = (t, units / t / 1e6)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_world_size_2():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
        assert all(p.exitcode == 0 for p in ps)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.5            # the slowest rank's time on every rank
    assert res[0][1] == pytest.approx(60000 / 1.5 / 1e6)   # whole-job units / slowest time


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 2.25, "cpu") == 2.25


def test_reference_arm_runs_on_rank_0_only(capsys):
    """Under torchrun the oracle arm prints nothing and does no work on ranks
    other than 0 (and needs no process group to do so)."""
    sys.path.insert(0, ROOT)
    import bench
    args = type("A", (), dict(workload="anode3d_256x128x128", steps=2, warmup=3, precision="fp32"))()
    assert bench.main_reference(args, 2, 1) == 0
    assert capsys.readouterr().out == ""


def test_oracle_on_all_cores_covers_the_workload(capsys):
    """The CPU baseline splits the workload's z-planes over processes (spawned,
    each a single-threaded oracle on its slab, periodic in z); together they
    cover every fluid cell, and the reference arm reports the core count."""
    sys.path.insert(0, ROOT)
    import json
    import bench
    from workloads import cases
    case = cases.anode_3d_small()
    cells, wall, procs, planes = bench.oracle_all_cores("anode3d_small", 2, 1, procs=2)
    assert procs == 2 and planes == case.solid.shape[0]
    assert cells == case.n_fluid and wall > 0
    args = type("A", (), dict(workload="anode3d_small", steps=2, warmup=1, precision="fp64",
                              oracle_procs=2, oracle_ttr=False, time_to_residual=1e-8,
                              max_steps=10))()
    assert bench.main_reference(args, 1, 0) == 0
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["cpu_baseline"]["cores"] == 2
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
