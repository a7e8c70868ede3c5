"""The multi-rank path without a GPU: two gloo ranks on the CPU.

The path shards by points (weak scaling): each rank hashes and indexes its
own shard, and the only collectives are the barrier and the max-over-ranks
of the step time.  Checked here: the helpers bench.py uses for the shard seed,
the job's time and throughput; that hashing shards separately and
concatenating equals hashing the whole (the points are independent), with the
oracle as the hasher on each rank; and that the library's top-k merge
(lsh_merge_topk, host code) of the ranks' per-shard query results, gathered
over gloo, equals the query over the whole database: a query's candidates in
the whole database are the union of its candidates in the shards.
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
    # sharded query: each rank indexes its 200 rows and answers 30 queries
    # (top-10 over its buckets); the library merges the gathered lists
    from paper_2503_06737_gb300 import lsh
    Q = X[::13][:30] + np.float32(0.05) * np.random.default_rng(5).standard_normal((30, 64)).astype(np.float32)
    _, _, _, qkeys = oracle.hash_dense(fam, Q, want_y=False, want_codes=False)
    idx = oracle.build_index(keys)
    lids, ldist, _ = oracle.query(idx, 64, X[lo:hi], Q, qkeys, 10, 0)
    ids_all = [torch.zeros((30, 10), dtype=torch.int32) for _ in range(world)]
    dist_all = [torch.zeros((30, 10), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(ids_all, torch.from_numpy(np.ascontiguousarray(lids, np.int32)))
    dist.all_gather(dist_all, torch.from_numpy(np.ascontiguousarray(ldist, np.float64)))
    if rank == 0:
        mids, mdist = lsh.merge_topk([t.numpy() for t in ids_all],
                                     [t.numpy().astype(np.float32) for t in dist_all], [0, 200])
        _, _, _, wkeys = oracle.hash_dense(fam, X, want_y=False, want_codes=False)
        wids, wdist, _ = oracle.query(oracle.build_index(wkeys), 64, X, Q, qkeys, 10, 0)
        ok = np.array_equal(mids, wids.astype(np.int64)) and np.array_equal(mdist, wdist.astype(np.float32))
        np.save(os.path.join(out_dir, "merge_ok.npy"), np.array([ok, (wids >= 0).sum() > 30]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch.distributed")
    if not dist.is_gloo_available():
        pytest.skip("gloo backend not built")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assert np.load(tmp_path / "ok.npy")[0]
    merge_ok, enough = np.load(tmp_path / "merge_ok.npy")
    assert enough  # the queries found candidates
    assert merge_ok
