"""Pins of the oracle's bucket key and of the family draws it uses.

Sec. 3.1 makes the concatenated m-code of a point the bucket of table t; the
paper defines no key.  The reading taken: for E2LSH kinds and SRP with m > 64,
a = sum_l code_l * ka_l mod 2^32, b = sum_l code_l * kb_l mod 2^32 (codes as
32-bit two's complement), key = a * 2^32 + b; for SRP with m <= 64 the key is
the bit pattern.  These tests restate that arithmetic with Python integers,
check hand-worked values, and restate the draws of the per-table multipliers
(and the rest of a count-sketch table) from SplitMix64's published definition,
so that a swapped ka/kb, a dropped mod 2^32 or a different sign extension of
the codes fails here.
"""
import numpy as np
import pytest

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def fold(codes, ka, kb):
    """The two multiply-add folds with Python integers (exact, then reduced)."""
    a = sum((int(c) & M32) * int(x) for c, x in zip(codes, ka)) & M32
    b = sum((int(c) & M32) * int(x) for c, x in zip(codes, kb)) & M32
    return (a << 32) | b


def mix64(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def stream(seed, t, count):
    st = mix64((seed + (t + 1) * GAMMA) & M64)
    out = []
    for _ in range(count):
        st = (st + GAMMA) & M64
        out.append(mix64(st))
    return out


def test_hand_worked_keys(orc):
    # m = 1, code -1: a = (2^32 - 1) * 3 mod 2^32 = 2^32 - 3, b = 2^32 - 5
    assert orc.key([-1], False, [3], [5]) == ((2**32 - 3) << 32) | (2**32 - 5)
    # INT32_MIN is 2^31 as an unsigned word; times an odd multiplier it stays 2^31
    assert orc.key([-2**31], False, [7], [9]) == (2**31 << 32) | 2**31
    # codes 2 and -3 with ka = (5, 7), kb = (11, 13): a = 10 - 21 = -11, b = 22 - 39 = -17
    assert orc.key([2, -3], False, [5, 7], [11, 13]) == ((2**32 - 11) << 32) | (2**32 - 17)
    # wrap: 2^31 - 1 twice with ka = 3: a = 6 (2^31 - 1) mod 2^32 = 2^32 - 6
    assert orc.key([2**31 - 1, 2**31 - 1], False, [3, 3], [1, 1]) == ((2**32 - 6) << 32) | (2**32 - 2)
    # the high word comes from ka, the low word from kb
    assert orc.key([1], False, [0xAAAAAAAB], [0x55555555]) == 0xAAAAAAAB55555555
    # SRP m <= 64: the bits themselves, bit l = code l
    assert orc.key([1, 0, 1, 1], True, [3] * 4, [5] * 4) == 0b1101
    assert orc.key([0] * 63 + [1], True, [3] * 64, [5] * 64) == 1 << 63


@pytest.mark.parametrize("m", [1, 7, 64, 65, 256])
def test_fold_restated_on_random_codes(orc, m):
    rng = np.random.default_rng(100 + m)
    for trial in range(50):
        codes = rng.integers(-2**31, 2**31, size=m, dtype=np.int64)
        codes[rng.random(m) < 0.2] = -2**31
        codes[rng.random(m) < 0.2] = rng.integers(-4, 5)
        ka = rng.integers(0, 2**32, size=m, dtype=np.uint64) | 1
        kb = rng.integers(0, 2**32, size=m, dtype=np.uint64) | 1
        assert orc.key(codes.astype(np.int32), False, ka, kb) == fold(codes, ka, kb)
        bits = (rng.random(m) < 0.5).astype(np.int32)
        want = fold(bits, ka, kb) if m > 64 else sum(int(v) << l for l, v in enumerate(bits))
        assert orc.key(bits, True, ka, kb) == want


@pytest.mark.parametrize("kind,m", [("cs_e2lsh", 16), ("hcs_e2lsh", 16), ("e2lsh", 8), ("cs_srp", 128),
                                    ("srp", 96)])
def test_pipeline_keys_restated(orc, kind, m):
    d, L, n = 48, 3, 20
    dims, mdims = ([6, 8], [4, 4]) if kind.startswith("hcs") else (None, None)
    f = orc.family(kind, d, m, L, w=0.5, seed=21, dims=dims, mdims=mdims)
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((n, d)) * 4).astype(np.float32)
    st, _, codes, keys = orc.hash_dense(f, X)
    assert st == 0
    assert (codes < 0).any() or orc.is_srp(f.kind)  # negative codes are exercised
    for i in range(n):
        for t in range(L):
            assert int(keys[t, i]) == fold(codes[i, t], f.ka[t], f.kb[t])


@pytest.mark.parametrize("m,d", [(16, 40), (12, 7)])
def test_count_sketch_tables_restated_from_splitmix(orc, m, d):
    """Bins, signs, offsets and key multipliers of a count-sketch table,
    restated from SplitMix64 (Steele, Lea and Flood 2014) and the draw order:
    d draws for (bin, sign), m draws for b, m draws for (ka, kb)."""
    seed, L, w = 987654321, 3, 2.5
    f = orc.family("cs_e2lsh", d, m, L, w=w, seed=seed)
    for t in range(L):
        r = stream(seed, t, d + 2 * m)
        bins = [((x >> 32) * m) >> 32 for x in r[:d]]
        signs = [-1 if (x >> 31) & 1 else 1 for x in r[:d]]
        b = [w * ((x >> 11) * 2.0 ** -53) for x in r[d:d + m]]
        ka = [(x >> 32) | 1 for x in r[d + m:]]
        kb = [(x & M32) | 1 for x in r[d + m:]]
        assert f.bins[t].tolist() == bins
        assert f.signs[t].tolist() == signs
        assert f.b[t].tolist() == b
        assert f.ka[t].tolist() == ka
        assert f.kb[t].tolist() == kb
