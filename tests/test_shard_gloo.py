"""Multi-process path on the CPU (gloo, world size 2): ticket sharding, the
tally sum over ranks and the job timing reduction.  Each rank transports its
share of the tickets with the oracle (no GPU here); the summed tallies must
equal one process transporting every ticket: bit-exact for the integer
tallies, to rounding for the floating-point ones."""

import os
import socket
import tempfile

import numpy as np
import pytest

import workloads
from paper_2411_14413_gb300.shard import ticket_shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tickets_to_ids(scene, begin, end):
    n = np.array([int(i["n"]) for i in scene.instances], dtype=np.int64)
    prefix = np.concatenate([[0], np.cumsum(n)])
    t = np.arange(begin, end, dtype=np.int64)
    inst = np.searchsorted(prefix, t, side="right") - 1
    return inst.astype(np.int32), (t - prefix[inst]).astype(np.uint64)


def _scene():
    return workloads.scene_quaternary(n_per_cathode=40)


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2411_14413_gb300.shard import combine_tallies, reduce_job

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = _scene()
        b, e = ticket_shard(sc.total_particles, rank, world)
        inst, pid = _tickets_to_ids(sc, b, e)
        o = oracle.OracleScene(sc).run_ids(inst, pid, n_threads=2)
        o["inst"] = inst
        tal = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in oracle.tally(sc, o).items()}
        tal["records"] = torch.zeros(3)  # per-particle buffers are not summed
        combine_tallies(tal)
        t, w = reduce_job(10.0 * (rank + 1), [e - b, 1.0])
        if rank == 0:
            np.savez(out_path, t=t, w=np.array(w), records=tal["records"].numpy(),
                     **{k: v.numpy() for k, v in tal.items() if k != "records"})
    finally:
        dist.destroy_process_group()


def test_ticket_shard_partitions_the_tickets():
    for n in [0, 1, 7, 100, 4_000_001]:
        for world in [1, 2, 3, 8]:
            shares = [ticket_shard(n, r, world) for r in range(world)]
            assert shares[0][0] == 0 and shares[-1][1] == n
            assert all(shares[i][1] == shares[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in shares]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ticket_shard(10, 2, 2)


def test_gloo_ranks_sum_to_the_single_process_tallies(oracle_mod):
    import torch.multiprocessing as mp

    world = 2
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "rank0.npz")
        mp.spawn(_worker, args=(world, _free_port(), path), nprocs=world, join=True)
        got = dict(np.load(path))
    sc = _scene()
    o = oracle_mod.OracleScene(sc).run_all(n_threads=2)
    o["inst"] = np.repeat(np.arange(len(sc.instances)), [int(i["n"]) for i in sc.instances])
    want = oracle_mod.tally(sc, o)
    for k in ("counts", "prim_counts", "timed_out"):
        assert np.array_equal(got[k], want[k]), k
    assert np.allclose(got["energy"], want["energy"], rtol=1e-12, atol=1e-9)
    assert int(got["prim_counts"].sum() + got["timed_out"].sum()) == sc.total_particles
    # the slowest rank's time and the work summed over ranks
    assert got["t"] == 20.0
    assert np.array_equal(got["w"], [sc.total_particles, 2.0])
    assert np.array_equal(got["records"], np.zeros(3))
