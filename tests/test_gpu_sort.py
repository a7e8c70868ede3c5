"""The table sort of Sec. 3.1's index (per table, (key, id) in key order with
ascending ids inside a bucket, cut into buckets) under each sort mode of
lsh_set_sort_mode: the global LSD passes and the bucket sort must both give
the oracle's arrays exactly.  The keys are seeded, made to reach every branch
of the bucket sort: buckets held on chip and buckets above its 5,120-key
capacity (through global memory), digits on which a table's or a bucket's
keys all agree (skipped passes), keys whose high bits never vary (the bucket
digit moves down), a single key value, and buckets of exactly the capacity
and one more."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import to_oracle
from paper_2503_06737_gb300 import lsh, workloads

pytestmark = pytest.mark.gpu

CAP = 5120  # keys of one bucket held on chip


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(autouse=True)
def _reset_mode():
    yield
    lsh.set_sort_mode(0)


def _u64(rng, shape):
    return rng.integers(0, 2**64, size=shape, dtype=np.uint64)


def key_sets():
    rng = np.random.default_rng(20250306)
    out = {}
    out["uniform_3x300k"] = _u64(rng, (3, 300000))
    # bit 63 and the low 48 bits vary: the bucket digit (bits 56-63) has two
    # values, so two buckets of about 50,000 keys each
    k = _u64(rng, (2, 100000))
    out["two_large_buckets"] = (k & np.uint64((1 << 48) - 1)) | (k & np.uint64(1 << 63))
    vals = _u64(rng, 5)
    out["five_values"] = vals[rng.integers(0, 5, size=(2, 50000))]
    out["one_value"] = np.full((1, 70000), np.uint64(0x0123456789ABCDEF), dtype=np.uint64)
    out["eleven_bit_keys"] = rng.integers(0, 2**11, size=(2, 200000), dtype=np.uint64)
    # bucket 0 (top byte 0) with exactly CAP and CAP + 1 keys
    n = 20000
    rows = []
    for B in (CAP, CAP + 1):
        k = _u64(rng, n) & np.uint64((1 << 56) - 1)
        top = rng.integers(1, 256, size=n, dtype=np.uint64)
        top[rng.permutation(n)[:B]] = 0
        rows.append(k | (top << np.uint64(56)))
    out["bucket_at_capacity"] = np.stack(rows)
    # top byte uniform, the low 56 bits from three values: per-bucket digits
    # that agree, others that differ
    low = _u64(rng, 3) & np.uint64((1 << 56) - 1)
    top = rng.integers(0, 256, size=(2, 150000), dtype=np.uint64)
    out["three_low_values"] = (top << np.uint64(56)) | low[rng.integers(0, 3, size=(2, 150000))]
    for n in (1, 2, 255, 4097, CAP + 1):
        out[f"tiny_{n}"] = _u64(rng, (3, n))
    out["full_table_1M"] = _u64(rng, (1, 1000000))
    return out


KEYS = key_sets()


@pytest.mark.parametrize("name", sorted(KEYS))
def test_sort_modes_match_oracle(name):
    keys_h = KEYS[name]
    L, n = keys_h.shape
    want = oracle.build_index(keys_h)
    lib = lsh.lib()
    keys = torch.from_numpy(keys_h.view(np.int64)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for mode in (1, 2, 0):
        lsh.set_sort_mode(mode)
        ids = torch.full((L, n), -1, dtype=torch.int32, device="cuda")
        ukeys = torch.zeros((L, n), dtype=torch.int64, device="cuda")
        offsets = torch.full((L, n + 1), -1, dtype=torch.int32, device="cuda")
        nb = torch.empty(L, dtype=torch.int64, device="cuda")
        st = lib.lsh_build_tables_static(_p(keys), n, L, _p(ids), _p(ukeys), _p(offsets), _p(nb), stream)
        assert st == 0, lib.lsh_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(nb.cpu().numpy(), want.nb), (name, mode)
        assert np.array_equal(ids.cpu().numpy().view(np.uint32), want.ids), (name, mode)
        gu = ukeys.cpu().numpy().view(np.uint64)
        go = offsets.cpu().numpy().view(np.uint32)
        for t in range(L):
            B = int(want.nb[t])
            assert np.array_equal(gu[t, :B], want.ukeys[t, :B]), (name, mode, t)
            assert np.array_equal(go[t, :B + 1], want.offsets[t, :B + 1]), (name, mode, t)


def test_index_above_bucket_limit_both_modes():
    # 1,200,000 rows: above the automatic bucket-sort limit (1,126,400), so
    # mode 0 takes the global passes and mode 2 the bucket sort; 8-wide rows
    # with m = 4 give many repeated keys (buckets above the on-chip capacity)
    n, d, m, L = 1200000, 8, 4, 2
    X = workloads.gmm(n, d, 16, seed=77, device="cpu")
    Xh, dt = to_oracle(X)
    ofam = oracle.family("cs_e2lsh", d, m, L, w=4.0, seed=5)
    _, _, _, okeys = oracle.hash_dense(ofam, Xh, dtype=dt, want_y=False, want_codes=False)
    want = oracle.build_index(okeys)
    fam = lsh.Family("cs_e2lsh", d, m, L, w=4.0, seed=5)
    Xd = X.cuda()
    for mode in (0, 2):
        lsh.set_sort_mode(mode)
        got = fam.build_index(Xd, keep_data=False).export()
        assert np.array_equal(got["nb"], want.nb), mode
        assert np.array_equal(got["ids"], want.ids), mode
        for t in range(L):
            B = int(want.nb[t])
            assert np.array_equal(got["ukeys"][t, :B], want.ukeys[t, :B]), (mode, t)
            assert np.array_equal(got["offsets"][t, :B + 1], want.offsets[t, :B + 1]), (mode, t)
    fam.close()
