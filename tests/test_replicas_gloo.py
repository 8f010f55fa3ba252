"""The N > 1 path on CPU: two gloo ranks, each stepping its own shard of the
cells (with the oracle, standing in for its GPU), max/sum over ranks, and the
gathered shards equal to the single-process result."""
import os
import socket

import numpy as np
import pytest

from paper_1110_4903_gb300 import replicas


def test_shard_ranges_cover_exactly():
    for n in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            cuts = [replicas.shard_range(n, r, world) for r in range(world)]
            assert cuts[0][0] == 0 and cuts[-1][1] == n
            assert all(cuts[i][1] == cuts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in cuts]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import oracle
    from paper_1110_4903_gb300 import synth
    w, r, _ = replicas.init("gloo")
    assert (w, r) == (world, rank)
    mech, f, dt = synth.workload("h2air-1k")
    a, b = replicas.shard_range(64, rank, world)
    fs = synth.subsample(f, np.arange(a, b))
    om = oracle.OracleMech(mech)
    rho, e = om.state_from_tpy(fs.T, fs.P, fs.Y)
    r1, e1, out = om.advance_batch(rho, e, dt, T_in=fs.T, opts=oracle.default_opts(max_halvings=0))
    np.save(os.path.join(out_dir, "rho_%d.npy" % rank), r1)
    mx = replicas.max_over_ranks(float(rank + 1))
    tot = replicas.sum_over_ranks(float(b - a))
    replicas.barrier()
    np.save(os.path.join(out_dir, "red_%d.npy" % rank), np.array([mx, tot]))
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    from paper_1110_4903_gb300 import synth
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.concatenate([np.load(tmp_path / ("rho_%d.npy" % r)) for r in range(world)], axis=1)
    for r in range(world):
        mx, tot = np.load(tmp_path / ("red_%d.npy" % r))
        assert mx == world and tot == 64
    mech, f, dt = synth.workload("h2air-1k")
    fs = synth.subsample(f, np.arange(64))
    om = oracle.OracleMech(mech)
    rho, e = om.state_from_tpy(fs.T, fs.P, fs.Y)
    r1, _, _ = om.advance_batch(rho, e, dt, T_in=fs.T, opts=oracle.default_opts(max_halvings=0))
    assert np.array_equal(got, r1)
