"""Host side of particle-sharded tracking, on CPU with two gloo ranks: the
collective adapter that Tracker.set_shard hands to the library
(paper_2208_02382_b300.torch_allreduce) and the split of a bunch over ranks.

What the library asks of the adapter: MIN and MAX of order-preserving int64
keys of doubles (the rest-frame extent of each rank's particles) must give the
keys of the global minimum and maximum, for negative and positive values
alike; SUM of the two fixed-point charge accumulators (hi = w >> 31 and
lo = w & (2^31 - 1) of 51-bit weights) must reproduce the charge of the whole
bunch exactly, whatever the split.  The keys and the split weights are formed
here in the test from their definitions."""
import multiprocessing as mp
import os
import socket
import struct
import tempfile

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def dkey(v: float) -> int:
    """Order-preserving signed 64-bit key of a double: its bit pattern, with
    the magnitude bits flipped for negative values."""
    b = struct.unpack("<q", struct.pack("<d", v))[0]
    return b if b >= 0 else b ^ 0x7FFFFFFFFFFFFFFF


def _rank_data(rank, world, n=20_001, nodes=4096):
    rng = np.random.default_rng(7)
    pos = rng.normal(0.0, 1e-3, size=(3, n))
    pos[2] *= 979.0                                   # long rest-frame bunch
    node = rng.integers(0, nodes, size=8 * n)
    w51 = rng.integers(0, 1 << 51, size=8 * n, dtype=np.int64)
    import paper_2208_02382_b300 as bt
    a, b = bt.shard_range(n, rank, world)
    sel = slice(8 * a, 8 * b)
    return pos, pos[:, a:b], node, node[sel], w51, w51[sel], nodes


def _accumulate(node, w51, nodes):
    hi = np.zeros(nodes, dtype=np.int64)
    lo = np.zeros(nodes, dtype=np.int64)
    np.add.at(hi, node, w51 >> 31)
    np.add.at(lo, node, w51 & ((1 << 31) - 1))
    return hi, lo


def _rank_main(rank, world, port, out):
    import datetime

    import torch
    import torch.distributed as dist

    import paper_2208_02382_b300 as bt
    from paper_2208_02382_b300 import _lib as L
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=60))
    red = bt.torch_allreduce()
    _, mine, _, node, _, w51, nodes = _rank_data(rank, world)
    big = np.iinfo(np.int64)
    kmin = [min((dkey(v) for v in mine[d]), default=big.max) for d in range(3)]
    kmax = [max((dkey(v) for v in mine[d]), default=big.min) for d in range(3)]
    tmin = torch.tensor(kmin, dtype=torch.int64)
    tmax = torch.tensor(kmax, dtype=torch.int64)
    red(tmin, L.BX_OP_MIN)
    red(tmax, L.BX_OP_MAX)
    hi, lo = _accumulate(node, w51, nodes)
    th, tl = torch.from_numpy(hi), torch.from_numpy(lo)
    red(th, L.BX_OP_SUM)
    red(tl, L.BX_OP_SUM)
    np.savez(out, kmin=tmin.numpy(), kmax=tmax.numpy(), hi=th.numpy(), lo=tl.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_allreduce_gives_the_global_extent_and_exact_charge():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        paths = [os.path.join(d, f"r{r}.npz") for r in range(2)]
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, paths[r])) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            if p.is_alive():
                p.kill()
                p.join()
        assert [p.exitcode for p in procs] == [0, 0]
        outs = [dict(np.load(q)) for q in paths]
    pos, _, node, _, w51, _, nodes = _rank_data(0, 1)
    for o in outs:                                    # every rank holds the same result
        assert o["kmin"].tolist() == [dkey(float(pos[d].min())) for d in range(3)]
        assert o["kmax"].tolist() == [dkey(float(pos[d].max())) for d in range(3)]
        hi, lo = _accumulate(node, w51, nodes)
        assert np.array_equal(o["hi"], hi) and np.array_equal(o["lo"], lo)
        # the charge itself: sum of all weights, recombined from hi and lo
        total = sum(int(h) << 31 for h in o["hi"]) + sum(int(x) for x in o["lo"])
        assert total == sum(int(x) for x in w51)


def test_key_order_matches_the_order_of_doubles():
    vals = [-np.inf, -1e300, -2.5, -1e-300, -0.0, 0.0, 1e-300, 3.0, 1e300, np.inf]
    keys = [dkey(v) for v in vals]
    assert keys == sorted(keys)
    assert dkey(-0.0) < dkey(0.0)


@pytest.mark.parametrize("n,world", [(10, 3), (0, 2), (1, 2), (25_000_000, 8)])
def test_shard_ranges_cover_the_bunch_once(n, world):
    import paper_2208_02382_b300 as bt
    rs = [bt.shard_range(n, r, world) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    sizes = [b - a for a, b in rs]
    assert max(sizes) - min(sizes) <= 1
