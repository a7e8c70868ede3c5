"""The continuous-batching serving loop (lsh_server_*): results equal lsh_query's
for the same queries, are the same alone and in any mix of concurrent
batches (bit for bit: each query is answered from its own row by its own CTA),
the same with and without captured graphs; batches overlap on the device
(several admitted at once) and a memory budget that fits one batch admits one
at a time; bad requests are refused on the host."""
import threading

import numpy as np
import pytest
import torch

from paper_2503_06737_gb300 import lsh, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    X = workloads.gmm(20000, 128, 64, seed=21, device="cpu", dtype=torch.float16).cuda()
    Q, _ = workloads.noisy_queries(X, 300, 0.05, seed=22)
    fam = lsh.Family("hcs_e2lsh", 128, 16, 16, w=4.0, seed=23, dims=[8, 16], mdims=[4, 4])
    idx = fam.build_index(X, keep_data=True)
    ref = idx.query(Q, k=10)
    torch.cuda.synchronize()
    return fam, idx, Q.cpu(), ref["ids"].cpu().numpy(), ref["dist"].cpu().numpy()


@pytest.mark.parametrize("use_graphs", [True, False])
def test_server_matches_query_alone_and_mixed(served, use_graphs):
    fam, idx, Q, rids, rdist = served
    srv = lsh.Server(idx, max_batch=256, slots=4, k=10, use_graphs=use_graphs)
    # alone: one query per request, each waited for before the next
    for i in range(0, 300, 37):
        ids, dist, lat = srv.wait(srv.submit(Q[i:i + 1]))
        assert np.array_equal(ids[0], rids[i]) and np.array_equal(dist[0], rdist[i])
        assert lat > 0
    # mixed: random batch sizes submitted from 3 threads without waiting
    rng = np.random.default_rng(int(use_graphs))
    cuts = np.sort(rng.choice(np.arange(1, 300), size=40, replace=False))
    parts = np.split(np.arange(300), cuts)
    got_ids = np.zeros_like(rids)
    got_dist = np.zeros_like(rdist)

    def worker(chunk):
        tickets = [(p, srv.submit(Q[p[0]:p[-1] + 1])) for p in chunk]
        for p, t in tickets:
            ids, dist, _ = srv.wait(t)
            got_ids[p] = ids
            got_dist[p] = dist

    th = [threading.Thread(target=worker, args=(parts[i::3],)) for i in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert np.array_equal(got_ids, rids) and np.array_equal(got_dist, rdist)
    st = srv.stats()
    assert st["completed_queries"] >= 300 and st["p99_ms"] >= st["p50_ms"] > 0
    assert st["admitted_peak"] >= 2  # batches overlapped on the device
    if use_graphs:
        assert st["graph_replays"] > 0 and st["graph_captures"] > 0
    srv.close()


def test_server_memory_budget_admission(served):
    fam, idx, Q, rids, _ = served
    per_row = 128 * 4 + 16 * 8 + 10 * 8
    one = 256 * per_row  # footprint of one largest batch (256-row bucket)
    # 150-query batches use the 256-row bucket: the budget admits one at a time
    srv = lsh.Server(idx, max_batch=256, slots=4, k=10, use_graphs=True, mem_budget=one)
    tickets = [srv.submit(Q[i * 150:(i + 1) * 150]) for i in range(2)] * 1
    tickets += [srv.submit(Q[:150]) for _ in range(2)]
    for i, t in enumerate(tickets):
        ids, _, _ = srv.wait(t)
        lo = (i * 150) if i < 2 else 0
        assert np.array_equal(ids, rids[lo:lo + 150])
    assert srv.stats(reset=True)["admitted_peak"] == 1
    # 50-query batches use the 64-row bucket: four fit in the same budget
    tickets = [srv.submit(Q[i * 50:(i + 1) * 50]) for i in range(6)]
    for i, t in enumerate(tickets):
        ids, _, _ = srv.wait(t)
        assert np.array_equal(ids, rids[i * 50:(i + 1) * 50])
    assert 1 <= srv.stats()["admitted_peak"] <= 4
    srv.close()


def test_server_rejects_bad_requests(served):
    fam, idx, Q, _, _ = served
    srv = lsh.Server(idx, max_batch=8, slots=1, k=5)
    with pytest.raises(lsh.LshError):
        srv.submit(Q[:9])  # more than max_batch
    with pytest.raises(lsh.LshError):
        lsh.Server(idx, max_batch=8, slots=1, k=5, mem_budget=16)  # budget below one batch
    srv.close()
    fam2 = lsh.Family("cs_e2lsh", 128, 16, 4)
    idx2 = fam2.build_index(workloads.iid(100, 128, device="cpu").cuda(), keep_data=False)
    with pytest.raises(lsh.LshError):
        lsh.Server(idx2, max_batch=8, slots=1, k=5)
