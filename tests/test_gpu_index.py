"""GPU parity of lsh_build_index (hash -> per-table stable radix sort of
(key, id) -> bucket segmentation) against the oracle's index of Sec. 3.1.

The ids, distinct keys, offsets and bucket counts must equal the oracle's
array for array (the oracle hashes the same rows itself).  Sizes span several
sort tiles (4096 keys) with ragged tails, many and few collisions, n = 0 and
n = 1; at the full 1,000,000-point size the invariants are checked on the
device (each table a permutation, keys non-decreasing along ids, offsets at
every key change) and the keys of sampled points are checked against the
oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_06737_gb300 import lsh, workloads

from gpu_helpers import to_oracle

pytestmark = pytest.mark.gpu


def _oracle_index(args, X):
    Xh, dt = to_oracle(X)
    ofam = oracle.family(args["kind"], args["d"], args["m"], args["L"], w=args.get("w", 4.0),
                         seed=args.get("seed", 42), dims=args.get("dims"), mdims=args.get("mdims"))
    st, _, _, keys = oracle.hash_dense(ofam, Xh, dtype=dt, want_y=False, want_codes=False)
    assert st == 0
    return oracle.build_index(keys)


@pytest.mark.parametrize("kind,n,d,m,L,w,dims,mdims", [
    ("cs_e2lsh", 10000, 128, 16, 10, 4.0, None, None),      # several sort tiles
    ("cs_srp", 9000, 128, 4, 6, 4.0, None, None),           # 16 buckets: heavy collisions
    ("hcs_e2lsh", 4097, 960, 64, 5, 4.0, [8, 10, 12], [4, 4, 4]),  # ragged last tile
    ("cs_e2lsh", 5000, 64, 2, 3, 64.0, None, None),         # very wide bins: few buckets
    ("hcs_srp", 1, 64, 8, 3, 4.0, [8, 8], [2, 4]),
    ("cs_e2lsh", 31, 32, 8, 40, 4.0, None, None),
])
def test_index_parity(kind, n, d, m, L, w, dims, mdims):
    args = dict(kind=kind, d=d, m=m, L=L, w=w, seed=17, dims=dims, mdims=mdims)
    X = workloads.iid(n, d, seed=n + d, device="cpu").cuda()
    fam = lsh.Family(**args)
    idx = fam.build_index(X, keep_data=False)
    got = idx.export()
    want = _oracle_index(args, X)
    assert np.array_equal(got["nb"], want.nb)
    assert np.array_equal(got["ids"], want.ids)
    for t in range(L):
        B = int(want.nb[t])
        assert np.array_equal(got["ukeys"][t, :B], want.ukeys[t, :B])
        assert np.array_equal(got["offsets"][t, :B + 1], want.offsets[t, :B + 1])


def test_index_empty():
    fam = lsh.Family("cs_e2lsh", 16, 4, 3)
    idx = fam.build_index(torch.empty((0, 16), device="cuda"), keep_data=False)
    n, nb = idx.info()
    assert n == 0 and (nb == 0).all()


def test_full_size_index_invariants():
    wl = workloads.WORKLOADS["gmm64_1M_d960"]
    n, L = wl["n"], wl["L"]
    X = workloads.gmm(n, wl["d"], wl["components"], seed=1235, device="cuda")
    args = dict(kind="hcs_e2lsh", d=960, m=64, L=L, w=4.0, seed=42, dims=wl["hcs_dims"],
                mdims=wl["hcs_mdims"])
    fam = lsh.Family(**args)
    keys = fam.hash(X, keys=True)["keys"]                 # [L, n] int64 view of u64
    idx = fam.build_index(X, keep_data=False)
    ex = idx.export()
    ids = torch.from_numpy(ex["ids"].astype(np.int64)).cuda()
    ar = torch.arange(n, device="cuda")
    for t in range(0, L, 7):
        it = ids[t]
        assert torch.equal(torch.sort(it).values, ar)     # a permutation
        k = keys[t][it].cpu().numpy().view(np.uint64)
        assert (k[1:] >= k[:-1]).all()                     # keys non-decreasing (unsigned)
        change = np.flatnonzero(k[1:] != k[:-1]) + 1
        B = int(ex["nb"][t])
        assert B == len(change) + 1
        assert np.array_equal(ex["offsets"][t, :B], np.concatenate([[0], change]).astype(np.uint32))
        assert ex["offsets"][t, B] == n
        assert np.array_equal(ex["ukeys"][t, :B], k[ex["offsets"][t, :B]])
        ii = ex["ids"][t]
        same = k[1:] == k[:-1]
        assert (ii[1:][same] > ii[:-1][same]).all()        # ids ascending inside a bucket
    # keys of sampled points equal the oracle's
    rows = np.random.default_rng(2).choice(n, 500, replace=False)
    Xs = X[torch.as_tensor(rows, device="cuda")]
    Xh, dt = to_oracle(Xs)
    ofam = oracle.family("hcs_e2lsh", 960, 64, L, w=4.0, seed=42, dims=wl["hcs_dims"], mdims=wl["hcs_mdims"])
    _, _, _, okeys = oracle.hash_dense(ofam, Xh, dtype=dt, want_y=False, want_codes=False)
    assert np.array_equal(keys[:, torch.as_tensor(rows, device="cuda")].cpu().numpy().view(np.uint64), okeys)


@pytest.mark.parametrize("keep", [False, True])
def test_rebuild_from_host_equals_device_rebuild(keep):
    """Host rows streamed in chunks (copies overlapping the hashing) give the
    same tables as a rebuild from the same rows on the device."""
    X = workloads.gmm(300_000, 128, 16, seed=51, device="cpu")
    Xh = X.pin_memory()
    fam = lsh.Family("cs_e2lsh", 128, 16, 8, w=4.0, seed=52)
    a = fam.build_index(X.cuda(), keep_data=keep)
    b = fam.build_index(workloads.gmm(300_000, 128, 16, seed=53, device="cuda"), keep_data=keep)
    b.rebuild_from_host(Xh, chunk_rows=70_000)  # ragged last chunk
    torch.cuda.synchronize()
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea["nb"], eb["nb"]) and np.array_equal(ea["ids"], eb["ids"])
    for t, nb in enumerate(ea["nb"]):  # the arrays hold nb[t] buckets; the rest is unused
        assert np.array_equal(ea["ukeys"][t, :nb], eb["ukeys"][t, :nb]), t
        assert np.array_equal(ea["offsets"][t, :nb + 1], eb["offsets"][t, :nb + 1]), t
    if keep:
        Q = X[:50].cuda() + 0.01
        ra, rb = a.query(Q, k=5), b.query(Q, k=5)
        assert torch.equal(ra["ids"], rb["ids"]) and torch.equal(ra["dist"], rb["dist"])
