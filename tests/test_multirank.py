"""Host logic of the multi-rank benchmark path on CPU (gloo, world size 2): every rank
runs its own independent query (own data seed, same shapes), timing is the max over
ranks, and the reported rate is the whole job's."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import argparse

    import bench
    wl = bench.workload(argparse.Namespace(workload="scale", scale=2e-6, w=65536), rank, device="cpu")
    ms_local = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    rate, ms_max = bench.whole_job_rate(wl.total_rows, ms_local, world)
    first_keys = wl.tables[0].cols[0][:16].tolist()
    out[rank] = (wl.total_rows, [t.n_rows for t in wl.tables], first_keys, rate, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    (rows0, shape0, keys0, rate0, ms0), (rows1, shape1, keys1, rate1, ms1) = out[0], out[1]
    assert shape0 == shape1 and rows0 == rows1            # same workload shape on every rank
    assert keys0 != keys1                                 # independent data per rank
    assert ms0 == ms1 == pytest.approx(15.0)              # max over ranks
    assert rate0 == rate1 == pytest.approx(rows0 * world / 0.015)
