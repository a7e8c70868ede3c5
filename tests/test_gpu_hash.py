"""GPU parity of lsh_hash (CS/HCS x E2LSH/SRP) against the FP64 oracle.

Codes and keys must match bit for bit; FP32 projections within 1e-5 relative
to max(|y|, ||x|| / sqrt(m)) (the FP32 value against the FP64 one).  Shapes
span several row tiles and table groups with ragged tails; the edge cases are
n = 0 and 1, d and n not multiples of 32, HCS zero padding, m = 1, L = 1,
m > 64 SRP (multi-word codes), non-finite rows, exact cancellation that the
FP32 path gets wrong and the FP64 recheck must repair, and the full-size
1,000,000 x 960 Gaussian-mixture workload on sampled rows.
"""
import numpy as np
import pytest
import torch

from paper_2503_06737_gb300 import lsh, workloads

pytestmark = pytest.mark.gpu

from gpu_helpers import compare_hash, compare_keys_only, to_oracle, unpack_bits  # noqa: E402


def _rows(n, d, seed, dtype=torch.float32, kind="iid"):
    if kind == "gmm":
        X = workloads.gmm(n, d, 16, seed=seed, device="cpu", dtype=dtype)
    else:
        X = workloads.iid(n, d, seed=seed, device="cpu", dtype=dtype)
    return X.cuda()


CASES = [
    # kind, n, d, m, L, dims, mdims, dtype
    ("cs_e2lsh", 1000, 128, 16, 10, None, None, torch.float32),
    ("cs_srp", 1000, 128, 16, 10, None, None, torch.float32),
    ("hcs_e2lsh", 700, 960, 64, 7, [8, 10, 12], [4, 4, 4], torch.float32),
    ("hcs_srp", 700, 960, 64, 7, [8, 10, 12], [4, 4, 4], torch.float32),
    ("cs_e2lsh", 333, 960, 64, 50, None, None, torch.float32),         # 3 table groups
    ("hcs_e2lsh", 257, 128, 16, 32, [8, 16], [4, 4], torch.float16),
    ("cs_e2lsh", 257, 128, 12, 32, None, None, torch.float16),
    ("cs_e2lsh", 300, 512, 32, 64, None, None, torch.bfloat16),
    ("hcs_e2lsh", 300, 512, 32, 64, [16, 32], [4, 8], torch.bfloat16),
    ("cs_srp", 77, 100, 256, 3, None, None, torch.float32),             # m > 64 SRP
    ("hcs_e2lsh", 45, 90, 16, 5, [8, 12], [4, 4], torch.float32),       # zero padding
    ("cs_e2lsh", 33, 37, 1, 1, None, None, torch.float32),              # m = 1, L = 1
    ("cs_srp", 1, 64, 64, 2, None, None, torch.float32),                # n = 1, m = 64
    ("hcs_srp", 129, 64, 8, 3, [4, 4, 4], [2, 2, 2], torch.float32),
    ("cs_e2lsh", 300, 200, 13, 7, None, None, torch.float32),           # m not a multiple of 4: scalar code stores
    ("hcs_srp", 150, 200, 26, 5, [10, 20], [2, 13], torch.float16),
]


@pytest.mark.parametrize("kind,n,d,m,L,dims,mdims,dtype", CASES)
def test_hash_parity(kind, n, d, m, L, dims, mdims, dtype):
    X = _rows(n, d, seed=n * 7 + d, dtype=dtype, kind="gmm" if d >= 512 else "iid")
    stats, rel = compare_hash(dict(kind=kind, d=d, m=m, L=L, w=4.0, seed=11, dims=dims, mdims=mdims), X)
    assert stats["n_entries"] == n * L * m
    assert stats["n_changed"] <= stats["n_flagged"]
    assert stats["n_nonfinite"] == 0 and stats["n_overflow"] == 0


@pytest.mark.parametrize("w", [0.05, 1.0, 64.0])
def test_hash_bin_widths(w):
    # narrow bins put many entries near an edge: exercises the FP64 recheck
    X = _rows(500, 128, seed=5)
    stats, _ = compare_hash(dict(kind="cs_e2lsh", d=128, m=16, L=8, w=w, seed=3), X)
    if w == 0.05:
        assert stats["n_flagged"] > 0


def test_strided_rows():
    base = _rows(200, 160, seed=9)
    X = base[:, :128]  # ld = 160 > d
    compare_hash(dict(kind="cs_srp", d=128, m=16, L=4, seed=5), X)


def test_empty_batch():
    fam = lsh.Family("cs_e2lsh", 64, 8, 4)
    out = fam.hash(torch.empty((0, 64), device="cuda"), codes=True, keys=True, stats=True)
    assert out["keys"].shape == (4, 0) and out["stats"]["n_entries"] == 0


def test_zero_and_duplicate_rows():
    X = _rows(100, 128, seed=6)
    X[10] = 0
    X[20] = X[30]
    compare_hash(dict(kind="cs_srp", d=128, m=16, L=6, seed=8), X)
    compare_hash(dict(kind="cs_e2lsh", d=128, m=16, L=6, seed=8), X)


def test_cancellation_repaired_by_recheck():
    """Pairs of +-1e8 terms that cancel exactly inside one bin wipe out the small
    terms summed before them in FP32; the FP64 recheck must restore the code."""
    d, m, L = 256, 8, 4
    fam_args = dict(kind="cs_srp", d=d, m=m, L=L, seed=21)
    tabs = lsh.sample_family_tables(**fam_args)
    rng = np.random.default_rng(0)
    X = (rng.standard_normal((64, d)) * 1e-3).astype(np.float32)
    h, s = tabs["bins"][0], tabs["signs"][0]
    for l in range(m):
        members = np.flatnonzero(h == l)
        pos = [j for j in members if s[j] > 0]
        neg = [j for j in members if s[j] < 0]
        if pos and neg:
            X[:, max(pos)] = 1e8   # the latest members of the bin cancel exactly
            X[:, max(neg)] = 1e8
    stats, _ = compare_hash(fam_args, torch.from_numpy(X).cuda(), check_proj=False)
    assert stats["n_flagged"] > 0
    assert stats["n_changed"] > 0  # the FP32 answer was wrong somewhere and got repaired


def test_nonfinite_rows_reported():
    X = _rows(64, 128, seed=12)
    X[5, 7] = float("nan")
    X[40, 0] = float("inf")
    fam = lsh.Family("cs_e2lsh", 128, 16, 4, seed=2)
    with pytest.raises(lsh.LshError) as e:
        fam.hash(X, keys=True, stats=True)
    assert e.value.status == 5  # LSH_ENONFINITE
    out = fam.hash(X, keys=True)  # without stats: sticky status word
    torch.cuda.synchronize()
    keys = out["keys"].cpu().numpy().view(np.uint64)
    assert (keys[:, 5] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    assert (keys[:, 40] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    assert fam.status() & 1
    assert fam.status() == 0  # cleared
    good = np.setdiff1d(np.arange(64), [5, 40])
    compare_hash(dict(kind="cs_e2lsh", d=128, m=16, L=4, seed=2), X[torch.as_tensor(good).cuda()])


def test_family_export_matches_sampler():
    args = dict(kind="hcs_e2lsh", d=960, m=64, L=5, w=4.0, seed=99, dims=[8, 10, 12], mdims=[4, 4, 4])
    fam = lsh.Family(**args)
    a = fam.export()
    b = lsh.sample_family_tables(**args)
    for k in ("bins", "signs", "b", "ka", "kb"):
        assert np.array_equal(a[k], b[k])


def test_deterministic_and_stream_ordered():
    X = _rows(4000, 128, seed=13)
    fam = lsh.Family("hcs_srp", 128, 16, 8, dims=[8, 16], mdims=[4, 4], seed=4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = fam.hash(X, keys=True, stream=s)["keys"]
    b = fam.hash(X, keys=True)["keys"]
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("kind", ["cs_e2lsh", "hcs_e2lsh", "cs_srp", "hcs_srp"])
def test_full_size_gist_like_sampled(kind):
    """1,000,000 x 960 64-component mixture, m = 64, L = 50 (HCS 8x10x12 -> 4x4x4):
    the whole batch is hashed in the launch configuration the bench times;
    2,000 sampled rows are checked against the oracle."""
    wl = workloads.WORKLOADS["gmm64_1M_d960"]
    X = workloads.gmm(wl["n"], wl["d"], wl["components"], seed=1235, device="cuda")
    hcs = kind.startswith("hcs")
    args = dict(kind=kind, d=960, m=64, L=50, w=4.0, seed=42,
                dims=wl["hcs_dims"] if hcs else None, mdims=wl["hcs_mdims"] if hcs else None)
    rows = np.sort(np.random.default_rng(1).choice(wl["n"], 2000, replace=False))
    rows = np.concatenate([rows, [0, wl["n"] - 1]])
    stats, rel = compare_hash(args, X, rows=rows)
    assert stats["n_entries"] == wl["n"] * 50 * 64
    del X
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kind,m,dims,mdims", [("hcs_e2lsh", 16, [8, 16], [4, 4]), ("cs_e2lsh", 12, None, None)])
def test_full_size_serving_rows_sampled(kind, m, dims, mdims):
    """10,000,000 x 128 FP16 rows of a 1,024-component mixture, L = 32, w = 48
    (the serving workload's index): the whole batch hashed keys-only in one
    call; 1,500 sampled rows and the first and last checked against the oracle."""
    import oracle
    wl = workloads.WORKLOADS["gmm1024_10M_d128_f16"]
    n, d, L = wl["n"], wl["d"], wl["L"]
    X = workloads.gmm(n, d, wl["components"], seed=1237, device="cuda", dtype=torch.float16)
    fam = lsh.Family(kind, d, m, L, w=48.0, seed=42, dims=dims, mdims=mdims)
    out = fam.hash(X, keys=True, stats=True)
    rows = np.concatenate([[0], np.sort(np.random.default_rng(5).choice(np.arange(1, n - 1), 1500, replace=False)),
                           [n - 1]])
    rt = torch.as_tensor(rows, device="cuda")
    of = oracle.family(kind, d, m, L, w=48.0, seed=42, dims=dims, mdims=mdims)
    Xs = X[rt].cpu().numpy()
    st, _, _, keys = oracle.hash_dense(of, Xs, want_y=False, want_codes=False)
    assert st == 0
    assert np.array_equal(out["keys"][:, rt].cpu().numpy().view(np.uint64), keys)
    assert out["stats"]["n_entries"] == n * m * L
    fam.close()
    del X, out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kind,d,m,L,dims,mdims,dtype", [
    ("cs_e2lsh", 128, 16, 8, None, None, torch.float32),
    ("hcs_e2lsh", 128, 16, 8, [8, 16], [4, 4], torch.bfloat16),
    ("cs_srp", 128, 16, 8, None, None, torch.float32),
    ("hcs_srp", 128, 16, 8, [8, 16], [4, 4], torch.float16),
    ("cs_srp", 100, 256, 3, None, None, torch.float32),     # multi-word SRP keys patched by sums
])
def test_deferred_recheck_patches(kind, d, m, L, dims, mdims, dtype):
    """Batches of 8192 rows or more queue their boundary bins for the recheck
    kernel, which patches codes, bits and keys; narrow bins (and SRP rows
    built to cancel) make many of them change."""
    X = _rows(9000, d, seed=31, dtype=dtype)
    w = 0.02 if "e2lsh" in kind else 4.0
    if "srp" in kind:
        X = torch.round(X * 1.5)  # small integers: many bins sum to exactly zero
    stats, _ = compare_hash(dict(kind=kind, d=d, m=m, L=L, w=w, seed=17, dims=dims, mdims=mdims), X)
    assert stats["n_flagged"] > 0


def test_deferred_recheck_repairs_cancellation():
    """The exact-cancellation rows of test_cancellation_repaired_by_recheck, in a
    batch large enough to take the queue: the patches must restore the bits."""
    d, m, L = 256, 8, 4
    fam_args = dict(kind="cs_srp", d=d, m=m, L=L, seed=21)
    tabs = lsh.sample_family_tables(**fam_args)
    rng = np.random.default_rng(1)
    X = (rng.standard_normal((9000, d)) * 1e-3).astype(np.float32)
    h, s = tabs["bins"][0], tabs["signs"][0]
    for l in range(m):
        members = np.flatnonzero(h == l)
        pos = [j for j in members if s[j] > 0]
        neg = [j for j in members if s[j] < 0]
        if pos and neg:
            X[:, max(pos)] = 1e8
            X[:, max(neg)] = 1e8
    stats, _ = compare_hash(fam_args, torch.from_numpy(X).cuda(), check_proj=False)
    assert stats["n_changed"] > 0


def test_deferred_recheck_queue_overflow():
    """Bins far narrower than the error bound flag nearly every entry: more
    than the queue holds, so the rest is rechecked inside the main kernel."""
    X = _rows(9000, 128, seed=32)
    stats, _ = compare_hash(dict(kind="cs_e2lsh", d=128, m=16, L=8, w=1e-5, seed=18), X)
    assert stats["n_flagged"] > 0.9 * 9000 * 128


# Every plan of the dense-row kernel computes the same codes: pin each shape
# (rows per lane, row groups, warps per table, tables per CTA, entry bytes)
# and check the keys-only and the full instantiations against the oracle.
PLANS = [(1, 1, 1, 4, 2, 0), (1, 1, 2, 50, 4, 0), (1, 2, 4, 8, 2, 0), (1, 4, 1, 3, 4, 0), (2, 1, 2, 6, 2, 0),
         (2, 1, 1, 16, 4, 0), (2, 2, 1, 5, 2, 0), (4, 1, 2, 4, 2, 0), (4, 1, 4, 2, 4, 0), (4, 1, 1, 32, 2, 0),
         (2, 1, 2, 8, 2, 1), (2, 1, 1, 50, 4, 1), (2, 2, 4, 3, 2, 1), (4, 1, 2, 6, 2, 1), (4, 2, 1, 4, 4, 1),
         (2, 4, 2, 2, 2, 1)]
PLAN_SHAPES = [
    # kind, d, m, L, dims, mdims, dtype
    ("cs_e2lsh", 960, 64, 13, None, None, torch.float32),
    ("hcs_srp", 200, 16, 9, [10, 20], [4, 4], torch.bfloat16),
    ("cs_srp", 300, 96, 5, None, None, torch.float16),
    ("hcs_e2lsh", 128, 16, 32, [8, 16], [4, 4], torch.float16),
]


def _pinned(plan, fn):
    lsh.set_sketch_plan(*plan)
    try:
        return fn()
    except lsh.LshError as e:
        assert e.status == 6, e  # LSH_EUNSUPPORTED: the pinned plan does not fit this shape
        return None
    finally:
        lsh.set_sketch_plan()


@pytest.mark.parametrize("plan", PLANS, ids=[str(p) for p in PLANS])
@pytest.mark.parametrize("kind,d,m,L,dims,mdims,dtype", PLAN_SHAPES, ids=[s[0] + str(s[1]) for s in PLAN_SHAPES])
def test_hash_every_plan(plan, kind, d, m, L, dims, mdims, dtype):
    fa = dict(kind=kind, d=d, m=m, L=L, w=4.0, seed=31, dims=dims, mdims=mdims)
    X = _rows(1000, d, seed=d + L, dtype=dtype, kind="gmm")
    _pinned(plan, lambda: compare_hash(fa, X))        # in-place rechecks, codes + proj + stats
    Xq = _rows(9001, d, seed=d + L + 1, dtype=dtype, kind="gmm")
    _pinned(plan, lambda: compare_keys_only(fa, Xq))  # queued rechecks, keys only
    Xu = _rows(301, d + 1, seed=d, dtype=dtype, kind="gmm")[:, 1:]  # rows not 16-byte aligned
    _pinned(plan, lambda: compare_keys_only(fa, Xu))


@pytest.mark.parametrize("kind,dims,mdims,dtype", [("cs_srp", None, None, torch.float32),
                                                   ("cs_e2lsh", None, None, torch.bfloat16),
                                                   ("hcs_e2lsh", [100, 100], [2, 4], torch.float32),
                                                   ("hcs_srp", [100, 100], [4, 2], torch.float16)])
def test_hash_long_rows(kind, dims, mdims, dtype):
    """Rows too long for the dense-row kernel's shared-memory tile (d = 10,000,
    the paper's Synthetic width) are hashed one warp per row in place, each bin
    bounded by its member count times max |x|."""
    fa = dict(kind=kind, d=10000, m=8, L=5, w=4.0, seed=9, dims=dims, mdims=mdims)
    X = _rows(150, 10000, seed=31, dtype=dtype, kind="iid")
    compare_hash(fa, X)
    compare_keys_only(fa, _rows(700, 10000, seed=32, dtype=dtype, kind="iid"))


@pytest.mark.parametrize("d,m,l,L,n,dtype", [(960, 64, 2, 7, 700, torch.float32), (128, 16, 4, 9, 9001, torch.float16),
                                            (300, 96, 3, 3, 500, torch.bfloat16), (64, 8, 8, 5, 129, torch.float32)])
def test_hash_csl_srp(d, m, l, L, n, dtype):
    """CSSRP-L (Table 1): each coordinate in l distinct bins of every table;
    codes and keys against the oracle (9,001 rows: queued rechecks), and
    with every plan shape pinned on the first case."""
    fa = dict(kind="csl_srp", d=d, m=m, L=L, seed=23, l=l)
    X = _rows(n, d, seed=d + l, dtype=dtype, kind="gmm")
    compare_hash(fa, X)
    compare_keys_only(fa, X)
    if d == 960:
        for plan in PLANS:
            _pinned(plan, lambda: compare_keys_only(fa, X))


def test_sketch_plan_query():
    """lsh_get_sketch_plan reports the pinned plan (with the balanced table
    group actually staged) and, unpinned, the default plan of a small batch."""
    fam = lsh.Family("cs_e2lsh", 960, 64, 13, w=4.0, seed=31)
    lsh.set_sketch_plan(2, 1, 2, 8, 2, 1)
    try:
        assert fam.sketch_plan(5000) == dict(rows_per_lane=2, row_groups=1, warps_per_table=2, tables_per_cta=7,
                                             entry_bytes=2, split_bins=1)
    finally:
        lsh.set_sketch_plan()
    p = fam.sketch_plan(5000)
    assert p["rows_per_lane"] * p["row_groups"] * (16 if p["split_bins"] else 32) == 32  # one 32-row tile
    assert p["tables_per_cta"] >= 1 and p["entry_bytes"] in (2, 4)
    fam.close()
