"""Pins of the oracle's index and query path against brute force.

The index is the set of L hash tables of Sec. 3.1: in table t every point sits
in the bucket of its key.  Invariants checked with plain Python dictionaries:
each id once per table, buckets ordered by key and ids ascending inside a
bucket, offsets monotone and ending at n.  The query (Sec. 6) takes the union
of the query's buckets and ranks it by exact distance; brute force over numpy
reproduces both the candidate set and the ranking, and the exact k-NN is the
ground truth of the recall.
"""
import numpy as np
import pytest


def _check_index(idx, keys):
    L, n = keys.shape
    for t in range(L):
        ids, uk, off = idx.table(t)
        assert sorted(ids.tolist()) == list(range(n))
        groups = {}
        for i in range(n):
            groups.setdefault(int(keys[t, i]), []).append(i)
        assert len(uk) == len(groups)
        assert (np.diff(uk.astype(object)) > 0).all() if len(uk) > 1 else True
        assert off[0] == 0 and off[-1] == n and (np.diff(off.astype(np.int64)) > 0).all()
        for bkt, k in enumerate(uk.tolist()):
            members = ids[off[bkt]:off[bkt + 1]].tolist()
            assert members == groups[k]  # ascending ids, exactly the points with that key


def test_index_small_random_keys(orc):
    rng = np.random.default_rng(1)
    keys = rng.integers(0, 20, size=(4, 300)).astype(np.uint64)  # many collisions
    keys[2] = rng.integers(0, 2 ** 63, size=300).astype(np.uint64) * 2 + 1
    keys[3] = 7
    _check_index(orc.build_index(keys), keys)


def test_index_from_hash(orc):
    d, m, L, n = 64, 4, 6, 500
    f = orc.family("cs_e2lsh", d, m, L, w=8.0, seed=2)
    X = np.random.default_rng(2).standard_normal((n, d)).astype(np.float32)
    _, _, codes, keys = orc.hash_dense(f, X, want_y=False)
    idx = orc.build_index(keys)
    _check_index(idx, keys)
    # points in one bucket share all m codes (the bucket of the concatenated code)
    for t in range(L):
        ids, uk, off = idx.table(t)
        for bkt in range(len(uk)):
            mem = ids[off[bkt]:off[bkt + 1]]
            assert (codes[mem, t] == codes[mem[0], t]).all()


def test_index_empty():
    import oracle
    idx = oracle.build_index(np.zeros((3, 0), np.uint64))
    assert (idx.nb == 0).all()


@pytest.mark.parametrize("metric", [0, 1])
def test_query_matches_brute_force(orc, metric):
    d, m, L, n, q, k = 32, 4, 5, 800, 25, 10
    kind = "cs_e2lsh" if metric == 0 else "cs_srp"
    f = orc.family(kind, d, m, L, w=6.0, seed=3)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n, d)).astype(np.float32)
    src = rng.integers(0, n, size=q)
    Q = (X[src] + 0.1 * rng.standard_normal((q, d))).astype(np.float32)
    _, _, _, keys = orc.hash_dense(f, X, want_y=False, want_codes=False)
    _, _, _, qkeys = orc.hash_dense(f, Q, want_y=False, want_codes=False)
    idx = orc.build_index(keys)
    ids, dist, ncand = orc.query(idx, d, X, Q, qkeys, k, metric)
    X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
    for i in range(q):
        cand = sorted({j for t in range(L) for j in range(n) if keys[t, j] == qkeys[t, i]})
        assert ncand[i] == len(cand)
        if metric == 0:
            dd = np.sqrt(((X64[cand] - Q64[i]) ** 2).sum(axis=1))
        else:
            dd = 1 - (X64[cand] @ Q64[i]) / (np.linalg.norm(X64[cand], axis=1) * np.linalg.norm(Q64[i]))
        order = sorted(range(len(cand)), key=lambda e: (dd[e], cand[e]))[:k]
        want_ids = [cand[e] for e in order] + [-1] * (k - len(order))
        assert ids[i].tolist() == want_ids
        np.testing.assert_allclose(dist[i, :len(order)], dd[order], rtol=1e-12, atol=1e-12)
        assert np.isinf(dist[i, len(order):]).all()
        # the query's own source point is found whenever it shares a bucket
        if src[i] in cand:
            assert src[i] in ids[i] or dist[i, -1] <= dd[cand.index(src[i])]


def test_bruteforce_knn(orc):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((300, 16)).astype(np.float32)
    Q = rng.standard_normal((7, 16)).astype(np.float32)
    ids, dist = orc.bruteforce_knn(X, Q, 5, 0)
    D = np.sqrt(((X.astype(np.float64)[None] - Q.astype(np.float64)[:, None]) ** 2).sum(-1))
    for i in range(7):
        want = np.lexsort((np.arange(300), D[i]))[:5]
        assert ids[i].tolist() == want.tolist()


def test_recall_near_duplicates(orc):
    # queries that are near copies of database points find them (recall of Sec. 6)
    d, m, L, n, q = 64, 8, 20, 2000, 40
    f = orc.family("cs_e2lsh", d, m, L, w=8.0, seed=5)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((n, d)).astype(np.float32)
    src = rng.integers(0, n, size=q)
    Q = (X[src] + 0.01 * rng.standard_normal((q, d))).astype(np.float32)
    _, _, _, keys = orc.hash_dense(f, X, want_y=False, want_codes=False)
    _, _, _, qkeys = orc.hash_dense(f, Q, want_y=False, want_codes=False)
    ids, _, _ = orc.query(orc.build_index(keys), d, X, Q, qkeys, 1, 0)
    assert (ids[:, 0] == src).mean() > 0.95
