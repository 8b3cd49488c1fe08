"""Multi-GPU is replicas only: every rank codes its own tensor, no collective
touches the data, and the job's time is the slowest rank's.  Checked here with
two gloo processes on CPU (the oracle stands in for each rank's codec)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2602_17849_gb300 import inputs
    x = inputs.make_e4m3("t4", 50_000, seed=rank).numpy()   # seed = rank, as bench.py does
    cont = oracle.encode(x, chunk_symbols=1024)
    st, y, _ = oracle.decode(cont)
    ms = 10.0 * (rank + 1)                                    # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms, world)
    dist.barrier()
    q.put((rank, ms_max, int(st), bool(np.array_equal(x, y)), int(cont.size), int(x[:64].sum())))
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [20.0, 20.0]                # max over ranks on both
    assert all(o[2] == 0 and o[3] for o in out)               # each replica round-trips
    assert out[0][5] != out[1][5]                             # and codes different data
    import bench
    assert bench.replica_throughput(2, 1 << 20, 2.0) == pytest.approx(2 * (1 << 20) / 2e-3 / 1e9)
