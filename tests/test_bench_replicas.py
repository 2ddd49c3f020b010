"""Host logic of the benchmark's N > 1 path, on CPU: the tracking step does not
shard (one bunch's kick needs the whole bunch's charge), so N GPUs run N
independent replicas and the job's throughput is all ranks' particle-steps
over the slowest rank's time.  These tests run that reduction over
torch.distributed with the gloo backend at world size 2, and check that the
reference arm's other ranks exit without work or output."""
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = (0.5, 0.8)[rank]
    units = (1.0e6, 3.0e6)[rank]
    s, u = bench.aggregate_replicas(seconds, units, dist, torch.device("cpu"))
    dist.barrier()
    queue.put((rank, s, u, bench.dist_env()))
    dist.destroy_process_group()


def test_replica_aggregation_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(queue.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, (r, seconds, units, env) in enumerate(got):
        assert r == rank
        assert seconds == 0.8            # the slowest rank
        assert units == 4.0e6            # all ranks' work
        assert env == (2, rank, rank)


def test_single_process_aggregation_is_identity():
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    assert bench.aggregate_replicas(1.25, 7.0) == (1.25, 7.0)


@pytest.mark.timeout(300)
def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=280, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
