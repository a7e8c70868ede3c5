"""The C ABI without a GPU: the library loads, exports every function that
include/lsh.h declares, its host-side family sampler draws exactly the
tables the oracle draws from the same seed, and invalid descriptions are
rejected on the host."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsh.h")


@pytest.fixture(scope="module")
def L():
    from paper_2503_06737_gb300 import build, lsh
    build.build()
    return lsh


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsh_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    lib = L.lib()
    names = declared_functions()
    assert len(names) >= 14
    for nm in names:
        assert hasattr(lib, nm), nm
    bound = {s[0] for s in L.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_version(L):
    assert b"sm_103a" in L.lib().lsh_version()


@pytest.mark.parametrize("kind,d,m,Lt,dims,mdims,seed", [
    ("cs_e2lsh", 128, 16, 10, None, None, 42),
    ("cs_srp", 20000, 256, 3, None, None, 43),
    ("hcs_e2lsh", 960, 64, 50, [8, 10, 12], [4, 4, 4], 44),
    ("hcs_srp", 20000, 256, 4, [100, 200], [16, 16], 45),
    ("hcs_e2lsh", 90, 16, 2, [8, 12], [4, 4], 46),
    ("e2lsh", 128, 16, 4, None, None, 47),
    ("srp", 64, 8, 3, None, None, 48),
])
def test_sampler_matches_oracle(L, orc, kind, d, m, Lt, dims, mdims, seed):
    a = L.sample_family_tables(kind, d, m, Lt, w=4.0, seed=seed, dims=dims, mdims=mdims)
    f = orc.family(kind, d, m, Lt, w=4.0, seed=seed, dims=dims, mdims=mdims)
    assert np.array_equal(a["b"], f.b)
    assert np.array_equal(a["ka"], f.ka) and np.array_equal(a["kb"], f.kb)
    if f.bins is not None:
        assert np.array_equal(a["bins"], f.bins) and np.array_equal(a["signs"], f.signs)
    if f.G is not None:
        assert np.array_equal(a["G"], f.G)


@pytest.mark.parametrize("bad", [
    dict(kind="cs_e2lsh", d=0, m=4, L=1),
    dict(kind="cs_e2lsh", d=8, m=0, L=1),
    dict(kind="cs_e2lsh", d=8, m=4, L=0),
    dict(kind="cs_e2lsh", d=8, m=4, L=1, w=0.0),
    dict(kind="cs_e2lsh", d=8, m=4, L=1, w=float("nan")),
    dict(kind="hcs_e2lsh", d=100, m=16, L=1, dims=[8, 12], mdims=[4, 4]),   # 96 < 100
    dict(kind="hcs_e2lsh", d=96, m=16, L=1, dims=[8, 12], mdims=[4, 5]),    # 20 != 16
    dict(kind="cs_srp", d=96, m=16, L=1, dims=[8, 12], mdims=[4, 4]),       # CS takes N = 1
    dict(kind=9, d=8, m=4, L=1),
])
def test_invalid_descriptions(L, bad):
    with pytest.raises(L.LshError) as e:
        L.sample_family_tables(**bad)
    assert e.value.status == 1  # LSH_EINVAL
    assert L.lib().lsh_last_error()


def test_null_arguments(L):
    import ctypes
    lib = L.lib()
    assert lib.lsh_make_family(None, None) == 1
    assert lib.lsh_hash(None, None, None, None, None, None, None) == 1
    assert lib.lsh_build_index(None, None, 0, None, None) == 1
    assert lib.lsh_query(None, None, 10, None, None, None, None) == 1
    assert lib.lsh_family_export(None, None, None, None, None, None, None) == 1
    assert lib.lsh_index_export(None, None, None, None, None) == 1
    assert lib.lsh_index_rebuild_host(None, None, 0, None) == 1
    lib.lsh_family_destroy(None)
    lib.lsh_index_destroy(None)


@pytest.mark.parametrize("kind", ["e2lsh", "srp"])
def test_bf16_family_matches_oracle(L, orc, kind):
    import torch
    a = L.sample_family_tables(kind, 512, 32, 4, seed=77, compute=1)
    f = orc.family(kind, 512, 32, 4, seed=77, compute=1)
    assert np.array_equal(a["G"], f.G)
    # the entries are the FP32 draws rounded to bfloat16 (ties to even), as torch rounds them
    g32 = orc.family(kind, 512, 32, 4, seed=77).G
    want = torch.from_numpy(g32).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(f.G, want)


def test_sketch_plan_pin_validation(L):
    """The plan pin is host-only: out-of-set values are refused, valid ones and
    the all-zero reset are accepted (no device needed)."""
    lib = L.lib()
    for args in [(3, 1, 1, 1, 2, 0), (4, 2, 1, 1, 2, 0), (1, 1, 3, 1, 2, 0), (1, 1, 1, 0, 2, 0),
                 (1, 1, 1, 4, 3, 0), (0, 1, 1, 1, 2, 0), (1, 1, 1, 1, 2, 1), (4, 4, 1, 1, 2, 1),
                 (2, 1, 1, 1, 2, 2)]:
        assert lib.lsh_set_sketch_plan(*args) == 1, args  # LSH_EINVAL
    for args in [(1, 4, 2, 25, 2, 0), (4, 1, 1, 8, 4, 0), (2, 2, 4, 1, 4, 0), (2, 1, 2, 8, 2, 1),
                 (4, 2, 1, 3, 4, 1), (2, 4, 4, 1, 2, 1)]:
        assert lib.lsh_set_sketch_plan(*args) == 0, args
    assert lib.lsh_set_sketch_plan(0, 0, 0, 0, 0, 0) == 0


def test_sort_mode_validation(L):
    """The sort-mode switch is host-only: 0, 1 and 2 are accepted, others refused."""
    lib = L.lib()
    for mode in (-1, 3, 7):
        assert lib.lsh_set_sort_mode(mode) == 1, mode  # LSH_EINVAL
    for mode in (1, 2, 0):
        assert lib.lsh_set_sort_mode(mode) == 0, mode


def test_merge_topk_against_restatement(L):
    """lsh_merge_topk (host only): the k best of the union by (distance,
    global id), from sorted per-shard lists with -1 / +inf tails; ties in
    distance across shards resolved by the global id."""
    import numpy as np
    rng = np.random.default_rng(3)
    for shards, q, k in ((1, 5, 4), (3, 40, 10), (4, 7, 1)):
        ids, dists, offs = [], [], []
        for s in range(shards):
            n_s = int(rng.integers(0, 2 * k))
            cand = rng.choice(50, size=min(n_s, 50), replace=False)
            dv = rng.integers(0, 6, size=(q, len(cand))).astype(np.float32) / 4  # many ties
            ii = np.full((q, k), -1, np.int32)
            dd = np.full((q, k), np.inf, np.float32)
            for i in range(q):
                order = sorted(range(len(cand)), key=lambda c: (dv[i, c], cand[c]))[:k]
                ii[i, :len(order)] = cand[order]
                dd[i, :len(order)] = dv[i, order]
            ids.append(ii)
            dists.append(dd)
            offs.append(1000 * s)
        got_i, got_d = L.merge_topk(ids, dists, offs)
        for i in range(q):
            pool = [(float(dists[s][i, j]), int(ids[s][i, j]) + offs[s]) for s in range(shards) for j in range(k)
                    if ids[s][i, j] >= 0]
            want = sorted(pool)[:k]
            want += [(float("inf"), -1)] * (k - len(want))
            assert [int(v) for v in got_i[i]] == [w[1] for w in want]
            assert [float(v) for v in got_d[i]] == [w[0] for w in want]
    assert L.lib().lsh_merge_topk(0, 1, 1, None, None, None, None, None) == 1  # LSH_EINVAL


@pytest.mark.parametrize("d,m,l", [(40, 16, 3), (960, 64, 2), (128, 8, 8)])
def test_csl_sampler_equals_oracle(L, d, m, l):
    """The library's CSSRP-L draws (l distinct bins per coordinate, by
    rejection) equal the oracle's independent draw."""
    import numpy as np
    import oracle
    t = L.sample_family_tables("csl_srp", d, m, 4, seed=17, l=l)
    o = oracle.family("csl_srp", d, m, 4, seed=17, l=l)
    for key in ("bins", "signs", "b", "ka", "kb"):
        assert np.array_equal(t[key], getattr(o, key)), key
