"""Particle-sharded tracking (bx_set_shard): one bunch split over two
processes, each with its own context and its share of the particles, which
exchange the box extent (MIN/MAX of integer keys) and the integer charge
accumulators (SUM) every kick through the allreduce callback.  The ranks run
as two processes on the same GPU with a gloo process group: the exchange goes
through host memory between kernel launches, so no kernel of one rank waits
on the other's.

The accumulators are exact integer sums, so the sharded coordinates must be
bitwise those of one process tracking the whole bunch (particles matched by
id), whatever the split: halves, a 1/3 - 2/3 split, and a rank holding no
particles at all.  They also match the oracle to 1e-11 relative."""
import multiprocessing as mp
import os
import socket
import tempfile

import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import track as tr
from tests.parity import REL_TOL, coord_rel_err, oracle_ref

pytestmark = pytest.mark.gpu

CASES = {
    # name: (workload, particles, kicks, grid, rebin interval, shares of rank 0 and 1)
    "fodo_halves": ("fodo_1e4_32", 9_001, 40, 16, 4, None),
    "fodo_third": ("fodo_1e4_32", 9_001, 40, 16, 4, 3_000),
    "fodo_empty_rank": ("fodo_1e4_32", 6_000, 25, 16, 8, 6_000),
    "chicane_128": ("chicane_25e6_128", 120_001, 6, 128, 4, None),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, out_path):
    import datetime

    import torch.distributed as dist

    import paper_2208_02382_b300 as bt
    name, npart, nk, n, rebin, first = CASES[case]
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=120))
    w = bg.workload(name)
    c = w.particles(npart)
    a, b = bt.shard_range(npart, rank, world) if first is None else \
        ((0, first) if rank == 0 else (first, npart))
    sp = bt.Species(w.species.mass_MeV, w.species.kinetic_MeV, w.species.charge_sign)
    coords = torch.tensor(np.ascontiguousarray(c[:, a:b]), dtype=torch.float64, device="cuda:0")
    ids = torch.arange(a, b, dtype=torch.int64, device="cuda:0")
    beam = bt.Beam(coords, sp, w.bunch_charge_C, ids=ids)
    trk = bt.Tracker(n, rebin_interval=rebin)
    trk.set_shard(bt.torch_allreduce(), npart)
    trk.track(beam, w.lattice, 0, nk // 2)
    trk.track(beam, w.lattice, nk // 2, nk - nk // 2)
    trk.sync()
    torch.cuda.synchronize()
    np.savez(out_path, coords=beam.coords.cpu().numpy(), ids=beam.ids.cpu().numpy(),
             log=np.array(trk.regrid_log(), dtype=np.int64))
    trk.close()
    dist.barrier()
    dist.destroy_process_group()


def _run_sharded(case, world=2):
    ctx = mp.get_context("spawn")
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        paths = [os.path.join(d, f"rank{r}.npz") for r in range(world)]
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, paths[r]))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=600)
        for p in procs:
            if p.is_alive():
                p.kill()
                p.join()
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        outs = [dict(np.load(q)) for q in paths]
    coords = np.concatenate([o["coords"] for o in outs], axis=1)
    ids = np.concatenate([o["ids"] for o in outs])
    assert np.array_equal(np.sort(ids), np.arange(len(ids)))
    return coords[:, np.argsort(ids)], [o["log"].tolist() for o in outs]


@pytest.mark.parametrize("case", list(CASES))
def test_sharded_tracking_is_bitwise_the_single_process_run(case):
    import paper_2208_02382_b300 as bt
    from paper_2208_02382_b300 import build
    build.build()
    name, npart, nk, n, rebin, _ = CASES[case]
    w = bg.workload(name)
    c = w.particles(npart)
    sharded, logs = _run_sharded(case)
    # one process, the whole bunch (the default CUDA-graph path)
    sp = bt.Species(w.species.mass_MeV, w.species.kinetic_MeV, w.species.charge_sign)
    beam = bt.Beam(torch.tensor(c, dtype=torch.float64, device="cuda:0"), sp, w.bunch_charge_C)
    trk = bt.Tracker(n, rebin_interval=rebin)
    trk.track(beam, w.lattice, 0, nk // 2)             # the same two calls as the ranks
    trk.track(beam, w.lattice, nk // 2, nk - nk // 2)
    trk.sync()
    torch.cuda.synchronize()
    ids = beam.ids.cpu().numpy()
    single = beam.coords.cpu().numpy()[:, np.argsort(ids)]
    assert logs[0] == logs[1] == trk.regrid_log()
    assert np.array_equal(sharded, single)
    # and the oracle
    otr = tr.Tracker(oracle_ref(w.species), w.bunch_charge_C, n)
    want = otr.track(otr.track(c, w.lattice, 0, nk // 2), w.lattice, nk // 2, nk - nk // 2)
    assert otr.regrid_log == logs[0]
    assert coord_rel_err(sharded, want) <= REL_TOL
    trk.close()
