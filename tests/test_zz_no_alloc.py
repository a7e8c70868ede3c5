"""The allocation-free table build, lsh_build_tables_static, called through the
C ABI: for callers that cannot allocate device memory while they run (fixed
memory budgets, a framework allocator that owns the GPU, hot paths that must
not stall in an allocator).  Its tables must equal those of lsh_build_index
exactly (integer arrays) on two calls in a row -- the second call runs over
the scratch the first one left behind -- and requests beyond its static limit
must be refused with LSH_EINVAL.  This file sorts last so that a run stopping
at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_06737_gb300 import lsh, workloads

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_build_matches_build_index_on_two_calls():
    lib = lsh.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, L, kind, seed in ((20000, 10, "cs_e2lsh", 1), (4097, 40, "cs_srp", 2)):
        X = workloads.iid(n, 128, seed=seed, device="cpu").cuda()
        fam = lsh.Family(kind, 128, 16, L, w=4.0, seed=seed)
        keys = fam.hash(X, keys=True)["keys"]
        ids = torch.empty((L, n), dtype=torch.int32, device="cuda")
        ukeys = torch.empty((L, n), dtype=torch.int64, device="cuda")
        offsets = torch.empty((L, n + 1), dtype=torch.int32, device="cuda")
        nb = torch.empty(L, dtype=torch.int64, device="cuda")
        st = lib.lsh_build_tables_static(_p(keys), n, L, _p(ids), _p(ukeys), _p(offsets), _p(nb), stream)
        assert st == 0, lib.lsh_last_error()
        torch.cuda.synchronize()
        want = fam.build_index(X, keep_data=False).export()
        got_nb = nb.cpu().numpy()
        assert np.array_equal(got_nb, want["nb"])
        assert np.array_equal(ids.cpu().numpy().view(np.uint32), want["ids"])
        gu = ukeys.cpu().numpy().view(np.uint64)
        go = offsets.cpu().numpy().view(np.uint32)
        for t in range(L):
            B = int(want["nb"][t])
            assert np.array_equal(gu[t, :B], want["ukeys"][t, :B])
            assert np.array_equal(go[t, :B + 1], want["offsets"][t, :B + 1])
        fam.close()


def test_static_build_refuses_oversize():
    lib = lsh.lib()
    n, L = (1 << 20) + 1, 1
    dummy = torch.empty(8, dtype=torch.int64, device="cuda")
    st = lib.lsh_build_tables_static(_p(dummy), n, L, _p(dummy), _p(dummy), _p(dummy), _p(dummy), None)
    assert st == 1  # LSH_EINVAL, before any device work
    assert b"LSH_STATIC_MAX_PAIRS" in lib.lsh_last_error()
    # within 2^20 pairs, but the digit histograms of 16,384 one-tile tables
    # take the scratch past 24 MiB
    st = lib.lsh_build_tables_static(_p(dummy), 64, 16384, _p(dummy), _p(dummy), _p(dummy), _p(dummy), None)
    assert st == 1
    assert b"24 MiB" in lib.lsh_last_error()
