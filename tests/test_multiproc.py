"""The multi-rank path without a GPU: two gloo ranks on the CPU.

The path shards by points (weak scaling): each rank hashes and indexes its
own shard, and the only collectives are the barrier and the max-over-ranks
of the step time.  Checked here: the helpers bench.py uses for the shard seed,
the job's time and throughput; and that hashing shards separately and
concatenating equals hashing the whole (the points are independent), with the
oracle as the hasher on each rank.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2503_06737_gb300 import workloads
    # the job's time is the slowest rank's, the throughput counts every rank's points
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    assert ms == 10.0 + 5.0 * (world - 1)
    assert bench.job_throughput(world, 1000, ms) == world * 1000 / (ms / 1e3)
    assert bench.shard_seed(rank) != bench.shard_seed(1 - rank)
    # each rank hashes its half of one dataset; rank 0 gathers and compares
    X = workloads.gmm(400, 64, 4, seed=99, device="cpu").numpy()
    fam = oracle.family("cs_e2lsh", 64, 8, 6, w=4.0, seed=3)
    lo, hi = rank * 200, (rank + 1) * 200
    _, _, _, keys = oracle.hash_dense(fam, X[lo:hi], want_y=False, want_codes=False)
    parts = [torch.zeros((6, 200), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(keys.view(np.int64).copy()))
    if rank == 0:
        _, _, _, whole = oracle.hash_dense(fam, X, want_y=False, want_codes=False)
        got = torch.cat(parts, dim=1).numpy().view(np.uint64)
        np.save(os.path.join(out_dir, "ok.npy"), np.array([np.array_equal(got, whole)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch.distributed")
    if not dist.is_gloo_available():
        pytest.skip("gloo backend not built")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assert np.load(tmp_path / "ok.npy")[0]
