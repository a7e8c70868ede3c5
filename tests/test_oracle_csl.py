"""Pins of the oracle's CSSRP-L (Table 1: a count-sketch projection matrix
with l nonzero entries in each column; the paper names it only by that
property).  Reading taken: coordinate i goes to l distinct bins, each with its
own random sign; the code is the sign of S x, as for CS-SRP (Definition 25).
Pinned here: the projection equals the explicit m x d matrix with l +-1
entries per column times x (exact on integer data); l = 1 reproduces the
count-sketch family and its keys; the draws restated from SplitMix64; the
moments E[y] = 0, Var[y] = l ||x||^2 / m; and the collision rate 1 - theta/pi.
"""
import numpy as np
import pytest

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix64(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def explicit_S(fam, t):
    """The m x d matrix of table t: S[h_r(i), i] = s_r(i) for r < l."""
    S = np.zeros((fam.m, fam.d))
    for i in range(fam.d):
        for r in range(fam.l):
            S[fam.bins[t, i * fam.l + r], i] += fam.signs[t, i * fam.l + r]
    return S


@pytest.mark.parametrize("d,m,l", [(50, 16, 3), (200, 64, 4), (7, 8, 8), (30, 5, 1)])
def test_projection_equals_explicit_matrix(orc, d, m, l):
    fam = orc.family("csl_srp", d, m, 3, seed=21, l=l)
    rng = np.random.default_rng(d + m + l)
    X = rng.integers(-50, 51, size=(6, d)).astype(np.float32)  # exact sums in FP64
    st, y, codes, keys = orc.hash_dense(fam, X)
    assert st == 0
    for t in range(3):
        S = explicit_S(fam, t)
        # l distinct rows per column: every column holds exactly l entries of +-1
        assert (np.abs(S) == 1).sum(axis=0).tolist() == [l] * d
        assert np.array_equal(y[:, t, :], X.astype(np.float64) @ S.T)
        assert np.array_equal(codes[:, t, :], (y[:, t, :] > 0).astype(np.int32))


def test_l1_is_the_count_sketch(orc):
    a = orc.family("csl_srp", 300, 32, 4, seed=77, l=1)
    b = orc.family("cs_srp", 300, 32, 4, seed=77)
    assert np.array_equal(a.bins, b.bins) and np.array_equal(a.signs, b.signs)
    assert np.array_equal(a.ka, b.ka) and np.array_equal(a.kb, b.kb)
    X = np.random.default_rng(1).standard_normal((20, 300)).astype(np.float32)
    assert np.array_equal(orc.hash_dense(a, X)[3], orc.hash_dense(b, X)[3])


def test_draws_restated_from_splitmix(orc):
    seed, d, m, l, L = 123, 25, 8, 3, 2
    fam = orc.family("csl_srp", d, m, L, seed=seed, l=l)
    for t in range(L):
        st = mix64((seed + (t + 1) * GAMMA) & M64)

        def nxt():
            nonlocal st
            st = (st + GAMMA) & M64
            return mix64(st)

        bins, signs = [], []
        for i in range(d):
            chosen = []
            for r in range(l):
                while True:
                    u = nxt()
                    bn = ((u >> 32) * m) >> 32
                    if bn not in chosen:
                        break
                chosen.append(bn)
                bins.append(bn)
                signs.append(-1 if (u >> 31) & 1 else 1)
        ka = []
        for q in range(m):
            nxt()  # the offsets b
        for q in range(m):
            ka.append((nxt() >> 32) | 1)
        assert fam.bins[t].tolist() == bins
        assert fam.signs[t].tolist() == signs
        assert fam.ka[t].tolist() == ka


def test_moments(orc):
    """Over many tables: E[y_b] = 0 and E[y_b^2] = l ||x||^2 / m (each
    coordinate lands in l of the m bins with a random sign)."""
    d, m, l, L = 64, 16, 4, 4000
    fam = orc.family("csl_srp", d, m, L, seed=9, l=l)
    x = np.random.default_rng(2).standard_normal((1, d)).astype(np.float32)
    _, y, _, _ = orc.hash_dense(fam, x)
    v = y[0].ravel()
    n2 = float((x.astype(np.float64) ** 2).sum())
    assert abs(v.mean()) < 5 * np.sqrt(l * n2 / m / v.size)
    assert abs(v.var() - l * n2 / m) < 5 * (l * n2 / m) * np.sqrt(2.0 / v.size) * 1.5


def test_collision_rate_matches_srp(orc):
    """Per-bit collision probability of two vectors at angle theta tends to
    1 - theta / pi (the SRP rate) for large d."""
    d, m, l, L = 4000, 16, 3, 400
    rng = np.random.default_rng(4)
    u = rng.standard_normal(d)
    w = rng.standard_normal(d)
    v = 0.8 * u + 0.6 * (w - (w @ u) / (u @ u) * u) * np.linalg.norm(u) / np.linalg.norm(w - (w @ u) / (u @ u) * u)
    theta = np.arccos(u @ v / np.linalg.norm(u) / np.linalg.norm(v))
    fam = orc.family("csl_srp", d, m, L, seed=13, l=l)
    _, _, c, _ = orc.hash_dense(fam, np.stack([u, v]).astype(np.float32))
    rate = float((c[0] == c[1]).mean())
    p = 1 - theta / np.pi
    sd = np.sqrt(p * (1 - p) / (m * L))
    assert abs(rate - p) < 5 * sd + 0.01, (rate, p)
