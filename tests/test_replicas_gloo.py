"""The N > 1 bench path on CPU: world_size-2 gloo ranks run the same
aggregation bench.py uses for its replicas (the time of the whole job is the
slowest rank's; throughput counts every rank's cells), and a bench process
launched the way the driver launches N > 1 (RANK/WORLD_SIZE in the
environment) prints exactly one line, from rank 0, on the reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_q):
    import torch.distributed as td

    import bench
    td.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                          world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], td, "cpu")
        g = bench.replica_throughput(world, 1000, 10, t)
        out_q.put((rank, t, g))
    finally:
        td.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    times = [0.25, 0.5]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, t, g in got:
        assert t == 0.5  # every rank sees the slowest rank's time
        assert g == pytest.approx(2 * 1000 * 10 / 0.5 / 1e9)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(0.125, None, "cpu") == 0.125
    assert bench.replica_throughput(1, 2097152, 20000, 1.0) == pytest.approx(41.94304)


def test_reference_arm_prints_only_on_rank_0(tmp_path):
    """Rank 1 of a 2-rank launch of the reference arm exits 0 without work
    or output; rank 0 prints one JSON line with impl=reference."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
