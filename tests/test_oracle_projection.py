"""Pins of the oracle's projections against what the paper fixes.

* Count sketch (Definition 4) is the product of x with the m x d matrix S that
  has the single entry s(i) in row h(i) of column i (Sec. 1 and 2 describe it
  as a projection with one nonzero per column).
* HCS (Definition 5) with N = 1 is a count sketch; with N = 2 it is
  S_1 P S_2^T for the d_1 x d_2 reshaping P of x (Sec. 1); for general N it
  is the Kronecker product (S_N (x) ... (x) S_1) applied to x, with the
  first-mode-fastest index maps of Definitions 5 and 19.
* Brute force on tiny inputs: the sums of Definitions 4/5 written as pure
  Python loops over every index tuple.
* Dense projection (Definitions 2/3): x G in FP64.
* Sparse rows give the same hash as their dense expansion.
* Exact widening of bf16 / f16 / e4m3 inputs matches the library decoders of
  numpy / torch.
"""
import itertools

import numpy as np
import pytest
import torch


def sketch_matrix(h, s, m):
    d = len(h)
    S = np.zeros((m, d))
    S[np.asarray(h), np.arange(d)] = np.asarray(s, np.float64)
    return S


@pytest.mark.parametrize("d,m", [(7, 3), (128, 16), (960, 64), (1000, 12)])
def test_cs_equals_sparse_matrix(orc, d, m):
    f = orc.family("cs_e2lsh", d, m, 3, seed=d + m)
    rng = np.random.default_rng(1)
    for t in range(3):
        S = sketch_matrix(f.bins[t], f.signs[t], m)
        assert (np.abs(S).sum(axis=0) == 1).all()  # one nonzero per column
        for _ in range(3):
            x = rng.standard_normal(d)
            np.testing.assert_allclose(orc.cs_project(x, f.bins[t], f.signs[t], m), S @ x,
                                       rtol=1e-12, atol=1e-12)


def test_hcs_n1_is_cs(orc):
    d, m = 300, 16
    f = orc.family("cs_e2lsh", d, m, 4, seed=2)
    rng = np.random.default_rng(2)
    for t in range(4):
        x = rng.standard_normal(d)
        a = orc.cs_project(x, f.bins[t], f.signs[t], m)
        b = orc.hcs_project(x, [d], [m], f.bins[t], f.signs[t])
        assert np.array_equal(a, b)


@pytest.mark.parametrize("d1,d2,m1,m2", [(8, 16, 4, 4), (100, 200, 16, 16), (5, 7, 2, 3)])
def test_hcs_n2_is_two_sided_product(orc, d1, d2, m1, m2):
    f = orc.family("hcs_e2lsh", d1 * d2, m1 * m2, 3, dims=[d1, d2], mdims=[m1, m2], seed=4)
    rng = np.random.default_rng(3)
    for t in range(3):
        (h1, s1), (h2, s2) = f.mode_tables(t)
        S1 = sketch_matrix(h1, s1, m1)
        S2 = sketch_matrix(h2, s2, m2)
        x = rng.standard_normal(d1 * d2)
        P = x.reshape(d2, d1).T          # P[i1, i2] = x[i1 + d1 * i2]
        Y = S1 @ P @ S2.T                # Y[l1, l2]
        want = Y.T.reshape(-1)           # vec: l = l1 + m1 * l2
        got = orc.hcs_project(x, [d1, d2], [m1, m2], [h1, h2], [s1, s2])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims,mdims", [([8, 10, 12], [4, 4, 4]), ([3, 4, 5, 2], [2, 3, 2, 2])])
def test_hcs_general_is_kronecker(orc, dims, mdims):
    d = int(np.prod(dims))
    m = int(np.prod(mdims))
    f = orc.family("hcs_srp", d, m, 2, dims=dims, mdims=mdims, seed=6)
    rng = np.random.default_rng(4)
    for t in range(2):
        mats = [sketch_matrix(h, s, mk) for (h, s), mk in zip(f.mode_tables(t), mdims)]
        K = np.ones((1, 1))
        for Sk in mats:                   # K = S_N (x) ... (x) S_1
            K = np.kron(Sk, K)
        x = rng.standard_normal(d)
        got = orc.hcs_project(x, dims, mdims, [h for h, _ in f.mode_tables(t)],
                              [s for _, s in f.mode_tables(t)])
        np.testing.assert_allclose(got, K @ x, rtol=1e-12, atol=1e-12)


def test_hcs_equals_cs_with_derived_tables(orc):
    dims, mdims = [8, 10, 12], [4, 4, 4]
    d, m = 960, 64
    f = orc.family("hcs_e2lsh", d, m, 2, dims=dims, mdims=mdims, seed=8)
    rng = np.random.default_rng(5)
    for t in range(2):
        mt = f.mode_tables(t)
        h = np.zeros(d, np.int32)
        s = np.ones(d, np.int8)
        for j in range(d):
            i1, i2, i3 = j % 8, (j // 8) % 10, j // 80
            h[j] = mt[0][0][i1] + 4 * mt[1][0][i2] + 16 * mt[2][0][i3]
            s[j] = mt[0][1][i1] * mt[1][1][i2] * mt[2][1][i3]
        x = rng.standard_normal(d)
        # same terms, same ascending-j order per bin: bit-identical
        assert np.array_equal(orc.hcs_project(x, dims, mdims, f.bins[t], f.signs[t]),
                              orc.cs_project(x, h, s, m))


def test_hcs_zero_padding(orc):
    # d = 90 viewed as 8 x 12 = 96: coordinates 90..95 are zeros (Sec. 6)
    dims, mdims = [8, 12], [4, 4]
    f = orc.family("hcs_e2lsh", 90, 16, 2, dims=dims, mdims=mdims, seed=10)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(90)
    xp = np.concatenate([x, np.zeros(6)])
    for t in range(2):
        a = orc.hcs_project(x, dims, mdims, f.bins[t], f.signs[t])
        b = orc.hcs_project(xp, dims, mdims, f.bins[t], f.signs[t])
        assert np.array_equal(a, b)


def _brute_hcs(x, dims, mdims, modes):
    """Definition 5 literally: for every bin tuple, sum over every index tuple."""
    N = len(dims)
    out = {}
    for ltuple in itertools.product(*[range(mk) for mk in mdims]):
        acc = 0.0
        for ituple in itertools.product(*[range(dk) for dk in dims]):
            if all(modes[k][0][ituple[k]] == ltuple[k] for k in range(N)):
                j = ituple[0]
                stride = 1
                for k in range(1, N):
                    stride *= dims[k - 1]
                    j += ituple[k] * stride
                sg = 1
                for k in range(N):
                    sg *= int(modes[k][1][ituple[k]])
                acc += sg * (x[j] if j < len(x) else 0.0)
        l = ltuple[0]
        stride = 1
        for k in range(1, N):
            stride *= mdims[k - 1]
            l += ltuple[k] * stride
        out[l] = acc
    return np.array([out[l] for l in range(len(out))])


@pytest.mark.parametrize("dims,mdims,d", [([8], [4], 8), ([2, 4], [2, 2], 8), ([2, 2, 2], [2, 1, 2], 7),
                                          ([3, 3], [2, 2], 9), ([4, 2], [4, 1], 6)])
def test_brute_force_tiny(orc, dims, mdims, d):
    m = int(np.prod(mdims))
    f = orc.family("hcs_e2lsh", d, m, 5, dims=dims, mdims=mdims, seed=12)
    # integer inputs keep every sum exact, so equality is exact
    rng = np.random.default_rng(7)
    for t in range(5):
        x = rng.integers(-9, 10, size=d).astype(np.float64)
        modes = f.mode_tables(t)
        want = _brute_hcs(x, dims, mdims, modes)
        got = orc.hcs_project(x, dims, mdims, [h for h, _ in modes], [s for _, s in modes])
        assert np.array_equal(got, want)


def test_dense_projection_is_matmul(orc):
    d, m, L = 128, 16, 10
    f = orc.family("e2lsh", d, m, L, seed=13)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((20, d)).astype(np.float32)
    st, y, codes, keys = orc.hash_dense(f, X)
    assert st == 0
    want = X.astype(np.float64) @ f.G.astype(np.float64)  # [n, m*L]
    np.testing.assert_allclose(y.reshape(20, m * L), want, rtol=1e-12, atol=1e-10)


def test_linearity(orc):
    d, m = 500, 16
    f = orc.family("cs_e2lsh", d, m, 1, seed=14)
    rng = np.random.default_rng(9)
    x, z = rng.standard_normal(d), rng.standard_normal(d)
    a, b = 1.5, -0.25
    lhs = orc.cs_project(a * x + b * z, f.bins[0], f.signs[0], m)
    rhs = a * orc.cs_project(x, f.bins[0], f.signs[0], m) + b * orc.cs_project(z, f.bins[0], f.signs[0], m)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", ["cs_e2lsh", "hcs_e2lsh", "cs_srp", "hcs_srp", "e2lsh", "srp"])
def test_pipeline_codes_and_keys(orc, kind):
    d, m, L = 96, 16, 4
    dims, mdims = ([8, 12], [4, 4]) if "hcs" in kind else (None, None)
    f = orc.family(kind, d, m, L, w=2.5, seed=15, dims=dims, mdims=mdims)
    rng = np.random.default_rng(10)
    X = rng.standard_normal((30, d)).astype(np.float32)
    st, y, codes, keys = orc.hash_dense(f, X)
    assert st == 0
    srp = orc.is_srp(f.kind)
    scale = np.sqrt(m) if kind in ("cs_e2lsh", "hcs_e2lsh") else 1.0
    if srp:
        assert np.array_equal(codes, (y > 0).astype(np.int32))
    else:
        assert np.array_equal(codes, np.floor((scale * y + f.b[None]) / f.w).astype(np.int32))
    for i in range(30):
        for t in range(L):
            assert keys[t, i] == orc.key(codes[i, t], srp, f.ka[t], f.kb[t])
    if srp:  # m <= 64: the key is the bit pattern
        for i in range(5):
            for t in range(L):
                assert int(keys[t, i]) == sum(int(codes[i, t, l]) << l for l in range(m))


def test_csr_equals_dense(orc):
    d, m, L, n = 2000, 32, 3, 40
    rng = np.random.default_rng(11)
    rows, cols, vals = [0], [], []
    dense = np.zeros((n, d), np.float32)
    for i in range(n):
        k = int(rng.integers(0, 50))
        c = np.sort(rng.choice(d, size=k, replace=False))
        v = rng.lognormal(size=k).astype(np.float32)
        dense[i, c] = v
        cols += list(c)
        vals += list(v)
        rows.append(len(cols))
    for kind, dims, mdims in [("cs_srp", None, None), ("hcs_srp", [40, 50], [4, 8]), ("cs_e2lsh", None, None)]:
        f = orc.family(kind, d, m, L, seed=16, dims=dims, mdims=mdims)
        a = orc.hash_csr(f, np.array(rows), np.array(cols, np.int32), np.array(vals, np.float32))
        b = orc.hash_dense(f, dense)
        assert a[0] == 0 and b[0] == 0
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_decoders(orc):
    h = np.arange(0, 65536, 97, dtype=np.uint16)
    f16 = h.view(np.float16).astype(np.float64)
    got = np.array([orc.from_f16(v) for v in h])
    ok = np.isfinite(f16)
    assert np.array_equal(got[ok], f16[ok])
    bf = torch.from_numpy(h.astype(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([orc.from_bf16(v) for v in h])
    ok = np.isfinite(bf)
    assert np.array_equal(got[ok], bf[ok])
    q = np.arange(256, dtype=np.uint8)
    e4 = torch.from_numpy(q).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([orc.from_e4m3(v) for v in q])
    ok = np.isfinite(e4)
    assert np.array_equal(got[ok], e4[ok])
    assert np.isnan(got[~ok]).all()


def test_round_e4m3_matches_torch_and_hand_values(orc):
    """The oracle's E4M3 rounding (written from the format) against torch's
    float8_e4m3fn conversion, and hand values: ties to even in the normal and
    subnormal ranges, carries into the next binade, saturation."""
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(20000), rng.standard_normal(2000) * 1e-2,
                        rng.uniform(-440, 440, 2000), np.ldexp(rng.integers(1, 64, 500), -10)]).astype(np.float32)
    want = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([orc.round_e4m3(float(x)) for x in v])
    assert np.array_equal(got, want)
    hand = {0.0: 0.0, 2.0 ** -10: 0.0, 3 * 2.0 ** -10: 2.0 ** -8, 2.0 ** -9: 2.0 ** -9,
            1.0625: 1.0, 1.1875: 1.25, 1.96875: 2.0, 240.0: 240.0, 248.0: 256.0, 447.0: 448.0,
            1000.0: 448.0, -1.0625: -1.0, 2.0 ** -6 + 2.0 ** -10: 2.0 ** -6}
    for x, y in hand.items():
        assert orc.round_e4m3(x) == y, (x, orc.round_e4m3(x), y)


def test_fp8_family_is_the_rounded_fp32_family(orc):
    f32 = orc.family("e2lsh", 64, 8, 3, seed=9)
    f8 = orc.family("e2lsh", 64, 8, 3, seed=9, compute=orc.E4M3)
    want = torch.from_numpy(f32.G).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    assert np.array_equal(f8.G, want)
    assert np.array_equal(f8.b, f32.b) and np.array_equal(f8.ka, f32.ka)


@pytest.mark.parametrize("kind", ["e2lsh", "srp", "cs_e2lsh", "hcs_srp"])
def test_fp8_rows_project_as_scale_times_projection(orc, kind):
    """A per-row-scaled FP8 row projects to scale x (projection of its FP8
    values): with small-integer FP8 values and an FP8 G the inner sums are
    exact, so y must equal scale * (Q @ G) (or * S q) bit for bit."""
    rng = np.random.default_rng(6)
    d, m, L, n = 32, 8, 2, 7
    dims = [4, 8] if kind.startswith("hcs") else None
    mdims = [2, 4] if dims else None
    fam = orc.family(kind, d, m, L, seed=12, dims=dims, mdims=mdims,
                     compute=orc.E4M3 if kind in ("e2lsh", "srp") else orc.F32)
    qv = rng.integers(-6, 7, size=(n, d)).astype(np.float32)
    q8 = torch.from_numpy(qv).to(torch.float8_e4m3fn)
    assert torch.equal(q8.to(torch.float32), torch.from_numpy(qv))
    scale = (rng.uniform(0.1, 3.0, n)).astype(np.float32)
    st, y, _, _ = orc.hash_dense(fam, q8.view(torch.uint8).numpy(), dtype=orc.E4M3, row_scale=scale)
    assert st == 0
    st0, y0, _, _ = orc.hash_dense(fam, qv, dtype=orc.F32)
    if kind in ("e2lsh", "srp"):
        ref = qv.astype(np.float64) @ fam.G.astype(np.float64)          # exact: small sums of FP8 products
        assert np.array_equal(y0.reshape(n, -1), ref)
    assert np.array_equal(y, scale.astype(np.float64)[:, None, None] * y0)
