"""GPU parity of the dense baselines E2LSH (Definition 2) and SRP (Definition 3):
FP32 SIMT GEMM with the fused epilogue and FP64 recheck against the oracle's
FP64 projection x G in ascending j.  Codes and keys bit-exact, projections
within 1e-5 of max(|y|, ||x||); shapes with ragged row / column tiles, tables
that straddle CTA tiles (m not dividing 128), f32/bf16/f16 inputs, and the
index and query path on dense kinds."""
import numpy as np
import pytest
import torch

from paper_2503_06737_gb300 import lsh, workloads

from gpu_helpers import compare_hash, compare_keys_only

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["e2lsh", "srp"])
@pytest.mark.parametrize("n,d,m,L,dtype", [
    (300, 128, 16, 10, torch.float32),
    (257, 960, 64, 3, torch.float32),
    (130, 37, 12, 13, torch.float32),   # 156 columns: tables straddle the 128-column tiles
    (200, 512, 32, 8, torch.bfloat16),
    (129, 128, 16, 4, torch.float16),
    (64, 100, 100, 2, torch.float32),   # SRP m > 64: two-word codes
])
def test_dense_parity(kind, n, d, m, L, dtype):
    X = workloads.gmm(n, d, 8, seed=n + d, device="cpu", dtype=dtype).cuda()
    stats, rel = compare_hash(dict(kind=kind, d=d, m=m, L=L, w=4.0, seed=13), X)
    assert stats["n_changed"] <= stats["n_flagged"]


@pytest.mark.parametrize("kind", ["e2lsh", "srp"])
def test_dense_fp32_queued_recheck(kind):
    """Batches of 8192 rows or more queue their boundary rechecks for a second
    kernel; narrow bins put many entries in the queue."""
    fa = dict(kind=kind, d=200, m=16, L=8, w=0.05, seed=3)
    X = workloads.gmm(9000, 200, 8, seed=7, device="cpu").cuda()
    stats, _ = compare_hash(fa, X, check_proj=False)
    assert stats["n_flagged"] > 0
    compare_keys_only(fa, X)


def test_dense_fp32_unaligned_rows():
    """Rows that do not start on 16 bytes are staged one value at a time."""
    X = workloads.gmm(300, 130, 8, seed=8, device="cpu").cuda()[:, 1:]
    compare_hash(dict(kind="e2lsh", d=129, m=16, L=5, seed=4), X)


def test_dense_narrow_bins_exercise_recheck():
    X = workloads.iid(200, 256, seed=3, device="cpu").cuda()
    stats, _ = compare_hash(dict(kind="e2lsh", d=256, m=16, L=8, w=0.01, seed=2), X)
    assert stats["n_flagged"] > 0


def test_dense_nonfinite_rows():
    X = workloads.iid(70, 64, seed=4, device="cpu").cuda()
    X[3, 5] = float("nan")
    fam = lsh.Family("e2lsh", 64, 16, 3, seed=1)
    with pytest.raises(lsh.LshError):
        fam.hash(X, keys=True, stats=True)
    k = fam.hash(X, keys=True)["keys"].cpu().numpy().view(np.uint64)
    assert (k[:, 3] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    good = torch.as_tensor(np.setdiff1d(np.arange(70), [3])).cuda()
    compare_hash(dict(kind="e2lsh", d=64, m=16, L=3, seed=1), X[good])


def test_dense_index_and_query():
    from test_gpu_query import _run
    X = workloads.gmm(4000, 64, 16, seed=6, device="cpu").cuda()
    Q, _ = workloads.noisy_queries(X, 20, 0.05, seed=9)
    _run(dict(kind="e2lsh", d=64, m=8, L=6, w=4.0, seed=5), X, Q, k=10)
    _run(dict(kind="srp", d=64, m=8, L=6, seed=5), X, Q, k=10)


@pytest.mark.parametrize("kind", ["e2lsh", "srp"])
@pytest.mark.parametrize("n,d,m,L", [(300, 512, 32, 8), (129, 128, 16, 16), (1000, 960, 64, 2), (77, 64, 8, 32),
                                     (700, 2048, 32, 8), (5000, 640, 16, 16)])  # d > 512: streamed row tiles
def test_dense_bf16_tensor_core_parity(kind, n, d, m, L):
    """BF16 rows and a BF16 family: the tcgen05 path (TMA, TMEM K-chunk
    accumulators, fused epilogue) against the oracle, bit-exact."""
    X = workloads.iid(n, d, seed=n + d, device="cpu", dtype=torch.bfloat16).cuda()
    args = dict(kind=kind, d=d, m=m, L=L, w=4.0, seed=31, compute=1)
    stats, rel = compare_hash(args, X)
    assert stats["n_changed"] <= stats["n_flagged"]


def test_dense_bf16_tensor_core_equals_simt_path():
    # strided rows (ld = 520, not a multiple of 8) take the SIMT path; both are exact
    X = workloads.iid(256, 520, seed=5, device="cpu", dtype=torch.bfloat16).cuda()
    fam = lsh.Family("e2lsh", 512, 32, 8, w=4.0, seed=3, compute=1)
    a = fam.hash(X[:, :512].contiguous(), codes=True, keys=True)
    b = fam.hash(X[:, :512], codes=True, keys=True)
    assert torch.equal(a["codes"], b["codes"]) and torch.equal(a["keys"], b["keys"])


@pytest.mark.parametrize("kind", ["e2lsh", "srp"])
def test_dense_bf16_tensor_core_many_tiles_per_cta(kind):
    """More output tiles than SMs: each persistent CTA walks several tiles
    through both TMEM accumulator buffers."""
    X = workloads.iid(20000, 128, seed=12, device="cpu", dtype=torch.bfloat16).cuda()
    compare_hash(dict(kind=kind, d=128, m=16, L=16, w=4.0, seed=8, compute=1), X)


@pytest.mark.parametrize("kind", ["e2lsh", "srp"])
def test_dense_bf16_tensor_core_wide_exponents(kind):
    """Rows whose coordinates span ~2^40 in magnitude: flagged entries there
    fail the fixed-point exactness condition (product exponents more than 37
    apart) and take the sequential FP64 loop."""
    X = workloads.iid(600, 256, seed=13, device="cpu", dtype=torch.float32)
    g = torch.Generator().manual_seed(5)
    X[::3] *= torch.exp2(torch.randint(-12, 13, X[::3].shape, generator=g).float())
    X = X.to(torch.bfloat16).cuda()
    compare_hash(dict(kind=kind, d=256, m=32, L=8, w=4.0, seed=9, compute=1), X)


def _grid_regimes(Xb, G):
    """For every (row, column): which exactness test of the recheck decides it.
    In units of 2^(least exponent of the row + least exponent of the column),
    the products are integers; 'one' = the magnitudes sum below 2^52, 'two' =
    they sum above 2^54 while every partial sum of the ascending loop stays
    below 2^52 (margins on both sides of 2^53 for the float64 estimates)."""
    def parts(T):
        h = T.view(torch.int16).numpy().astype(np.int64) & 0xFFFF
        e = (h >> 7) & 0xFF
        return (h & 0x7F) | (np.minimum(e, 1) << 7), np.maximum(e, 1) - 134, np.where(h >> 15, -1, 1)
    Mx, Ex, sx = parts(Xb)
    Mg, Eg, sg = parts(G)
    big = 1 << 20
    ex0 = np.where(Mx > 0, Ex, big).min(1)
    eg0 = np.where(Mg > 0, Eg, big).min(0)
    rx = np.where(Mx > 0, Ex, -big).max(1) - ex0
    rg = np.where(Mg > 0, Eg, -big).max(0) - eg0
    Xi = (sx * (Mx << np.maximum(Ex - ex0[:, None], 0))).astype(np.float64)
    Gi = (sg * (Mg << np.maximum(Eg - eg0[None, :], 0))).astype(np.float64)
    shape = (rx[:, None] <= 23) & (rg[None, :] <= 23) & (16 + rx[:, None] + rg[None, :] <= 53)
    mag = np.abs(Xi) @ np.abs(Gi)
    part = np.stack([np.abs(np.cumsum(Xi[r][:, None] * Gi, axis=0)).max(0) for r in range(Xi.shape[0])])
    return shape & (mag < 2.0**52), shape & (mag > 2.0**54) & (part < 2.0**52)


def test_dense_bf16_tensor_core_recheck_partial_sum_pass():
    """Rows of +-[1, 2) values with one coordinate near 2^-20: the products'
    magnitudes sum past 2^53 on the common exponent grid, so the one-pass
    exactness test fails, while the partial sums of the ascending loop stay
    below 2^53 -- the recheck's second pass proves them exact.  Bins narrower
    than the error bound flag every entry, more than the queue holds, so both
    the recheck kernel and the in-kernel recheck take this route."""
    import oracle
    n, d, m, L = 300, 512, 32, 8
    g = torch.Generator().manual_seed(21)
    X = (1 + torch.rand(n, d, generator=g)) * (2 * torch.randint(0, 2, (n, d), generator=g) - 1).float()
    X[torch.arange(n), torch.randint(0, d, (n,), generator=g)] = torch.exp2(-torch.randint(19, 23, (n,), generator=g).float())
    Xb = X.to(torch.bfloat16)
    args = dict(kind="e2lsh", d=d, m=m, L=L, w=1e-4, seed=4, compute=1)
    G = torch.from_numpy(oracle.family("e2lsh", d, m, L, w=1e-4, seed=4, compute=oracle.BF16).G).to(torch.bfloat16)
    one, two = _grid_regimes(Xb, G)
    assert two.mean() > 0.2 and one.mean() > 0.1, (two.mean(), one.mean())
    stats, _ = compare_hash(args, Xb.cuda())
    assert stats["n_flagged"] >= 0.9 * n * m * L


def test_dense_bf16_tensor_core_nonfinite_row():
    X = workloads.iid(300, 128, seed=14, device="cpu", dtype=torch.bfloat16).cuda()
    X[7, 100] = float("inf")
    fam = lsh.Family("e2lsh", 128, 16, 16, w=4.0, seed=2, compute=1)
    with pytest.raises(lsh.LshError):
        fam.hash(X, keys=True, stats=True)
    k = fam.hash(X, keys=True)["keys"].cpu().numpy().view(np.uint64)
    assert (k[:, 7] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    good = torch.as_tensor(np.setdiff1d(np.arange(300), [7])).cuda()
    compare_hash(dict(kind="e2lsh", d=128, m=16, L=16, w=4.0, seed=2, compute=1), X[good])


def test_dense_bf16_tensor_core_recheck_queue_overflow():
    """Bins narrower than the error bound flag every entry: more than the
    recheck queue holds, so part of them is rechecked inside the main kernel."""
    X = workloads.iid(300, 512, seed=15, device="cpu", dtype=torch.bfloat16).cuda()
    stats, _ = compare_hash(dict(kind="e2lsh", d=512, m=32, L=8, w=1e-4, seed=4, compute=1), X)
    assert stats["n_flagged"] >= 0.9 * 300 * 256


def _fp8_compare(kind, n, d, m, L, seed, X=None):
    """Per-row-scaled FP8 rows and an FP8 family: the tcgen05 kind::f8f6f4
    path against the oracle (projection = scale x projection of the E4M3
    values), codes and keys bit for bit, projections within 1e-5."""
    import oracle
    if X is None:
        X = workloads.iid(n, d, seed=seed, device="cpu")
    q, scale = workloads.fp8_rows(X)
    fam = lsh.Family(kind, d, m, L, w=4.0, seed=seed, compute=lsh.FP8_E4M3)
    out = fam.hash(q.cuda(), codes=True, keys=True, proj=True, stats=True, row_scale=scale.cuda())
    of = oracle.family(kind, d, m, L, w=4.0, seed=seed, compute=oracle.E4M3)
    st, y, codes, keys = oracle.hash_dense(of, q.numpy(), dtype=oracle.E4M3, row_scale=scale.numpy())
    assert st == 0
    gc = out["codes"].cpu().numpy()
    if fam.is_srp:
        from gpu_helpers import unpack_bits
        gc = unpack_bits(gc, m)
    assert np.array_equal(gc, codes), np.argwhere(gc != codes)[:5]
    assert np.array_equal(out["keys"].cpu().numpy().view(np.uint64), keys)
    gp = out["proj"].cpu().numpy().astype(np.float64)
    # the tolerance of every dense path: 1e-5 relative to max(|y|, ||x||), x = scale q
    xn = np.linalg.norm(q.view(torch.float8_e4m3fn).to(torch.float64).numpy(), axis=1) * scale.numpy()
    tol = np.maximum(np.abs(y), xn[:, None, None])
    assert np.all(np.abs(gp - y) <= 1e-5 * tol), float(np.max(np.abs(gp - y) / tol))
    fam.close()
    return out["stats"]


@pytest.mark.parametrize("kind", ["e2lsh", "srp"])
@pytest.mark.parametrize("n,d,m,L", [(300, 512, 32, 8), (129, 128, 16, 16), (1000, 1024, 64, 2), (20000, 256, 32, 8),
                                     (500, 2048, 16, 8)])  # d = 2048: the row tile streams its K slices
def test_dense_fp8_tensor_core_parity(kind, n, d, m, L):
    st = _fp8_compare(kind, n, d, m, L, seed=n + d)
    assert st["n_changed"] <= st["n_flagged"]


def test_dense_fp8_rows_with_tiny_and_zero_rows():
    X = workloads.iid(400, 256, seed=77, device="cpu")
    X[3] = 0
    X[5] *= 1e-30
    X[7] *= 1e4
    _fp8_compare("e2lsh", 400, 256, 16, 8, seed=5, X=X)


@pytest.mark.parametrize("compute", ["bf16", "fp8"])
def test_dense_tensor_core_full_size_sampled(compute):
    """4,000,000 x 512 i.i.d. rows, m = 32, L = 64 (GEMM 4M x 512 x 2048): the
    whole batch is hashed keys-only in one call, as the bench times it (BF16
    rows, or per-row-scaled FP8 rows); 1,500 sampled rows and the first and
    last are checked against the oracle bit for bit."""
    import oracle
    wl = workloads.WORKLOADS["iid_4M_d512_bf16"]
    n, d, m, L, w = wl["n"], wl["d"], wl["m"], wl["L"], wl["w"]
    X = workloads.iid(n, d, seed=1238, device="cuda", dtype=torch.bfloat16)
    rows = np.concatenate([[0], np.sort(np.random.default_rng(4).choice(np.arange(1, n - 1), 1500, replace=False)),
                           [n - 1]])
    rt = torch.as_tensor(rows, device="cuda")
    if compute == "bf16":
        fam = lsh.Family("e2lsh", d, m, L, w=w, seed=42, compute=lsh.BF16)
        out = fam.hash(X, keys=True, stats=True)
        Xs, dt, rs = X[rt].cpu().view(torch.int16).numpy().view(np.uint16), oracle.BF16, None
        of = oracle.family("e2lsh", d, m, L, w=w, seed=42, compute=oracle.BF16)
    else:
        q8, sc8 = workloads.fp8_rows(X)
        fam = lsh.Family("e2lsh", d, m, L, w=w, seed=42, compute=lsh.FP8_E4M3)
        out = fam.hash(q8, keys=True, stats=True, row_scale=sc8)
        Xs, dt, rs = q8[rt].cpu().numpy(), oracle.E4M3, sc8[rt].cpu().numpy()
        of = oracle.family("e2lsh", d, m, L, w=w, seed=42, compute=oracle.E4M3)
        del q8, sc8
    st, _, _, keys = oracle.hash_dense(of, Xs, dtype=dt, row_scale=rs, want_y=False, want_codes=False)
    assert st == 0
    assert np.array_equal(out["keys"][:, rt].cpu().numpy().view(np.uint64), keys)
    assert out["stats"]["n_entries"] == n * m * L
    assert out["stats"]["n_changed"] <= out["stats"]["n_flagged"]
    fam.close()
    del X, out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,d,L", [(700, 256, 3), (300, 960, 2), (9000, 512, 1)])
def test_dense_tensor_core_m128(n, d, L):
    """E2LSH with m = 128 on the tensor cores: one table fills a 128-column
    tile and its four 32-column slices combine their partial keys; BF16 and
    per-row-scaled FP8 rows against the oracle (9,000 rows: queued rechecks)."""
    X = workloads.iid(n, d, seed=n + d + 1, device="cpu", dtype=torch.bfloat16).cuda()
    stats, _ = compare_hash(dict(kind="e2lsh", d=d, m=128, L=L, w=4.0, seed=33, compute=1), X)
    assert stats["n_changed"] <= stats["n_flagged"]
    st = _fp8_compare("e2lsh", n, d, 128, L, seed=n + d + 2)
    assert st["n_changed"] <= st["n_flagged"]
