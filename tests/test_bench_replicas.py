"""Host logic of the benchmark, on CPU.  With N > 1 ranks the bench tracks one
bunch sharded over the ranks (each holds its share of the particles), and the
job's throughput is all ranks' particle-steps over the slowest rank's time.
These tests run that reduction over torch.distributed with the gloo backend at
world size 2, check that the reference arm's other ranks exit without work or
output, and that the CPU baseline's all-cores run of the oracle (its functions
over particle chunks in worker processes) tracks like the oracle itself."""
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


@pytest.mark.timeout(300)
def test_oracle_on_cores_tracks_like_the_oracle():
    """bench.OracleOnCores (two worker processes) against oracle.track.Tracker:
    the same regrid log and coordinates to rounding (the chunk grids are summed
    in chunk order, the only change of operation order)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import beamgen as bg
    from oracle import physics as ph
    from oracle import track as tr
    w = bg.workload("fodo_1e4_32")
    w.n_grid = 16
    c = w.particles(3001)
    sp = w.species
    t = tr.Tracker(ph.RefPart(sp.mass_MeV, sp.kinetic_MeV, sp.charge_sign), w.bunch_charge_C, 16)
    want = t.track(c, w.lattice, 0, 9)
    o = bench.OracleOnCores(w, c, 2)
    try:
        o.track(w.lattice, 0, 9)
        got = o.C.copy()
    finally:
        o.close()
    assert o.regrid_log == t.regrid_log
    rms = np.sqrt(np.mean(want ** 2, axis=1))[:, None]
    assert np.max(np.abs(got - want) / np.maximum(np.abs(want), rms)) < 1e-13
