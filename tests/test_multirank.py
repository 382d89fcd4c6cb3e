"""The multi-GPU path of the benchmark is replicas only: every rank runs its own chain (its own
seed) and the job's throughput is all ranks' trials over the slowest rank's time.  Checked with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.env_rank()
    total_ms = 100.0 + 50.0 * rank          # rank 1 is slower
    search_ms = 90.0 + 40.0 * rank
    res = bench.aggregate_ranks(dist, total_ms, search_ms, trials_local=1_000_000, device="cpu")
    out[rank] = (r, w, local, bench.replica_seed(rank)) + tuple(res)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_timing():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        r, w, local, seed, total_ms, search_ms, value = res[rank]
        assert (r, w, local) == (rank, 2, rank)
        assert total_ms == 150.0 and search_ms == 130.0      # max over ranks
        assert value == pytest.approx(2_000_000 / 0.150)      # all ranks' trials / slowest time
    assert res[0][3] != res[1][3]                            # independent chains
