"""The integer arithmetic the kernels rely on, checked on the host.

* Quotients by a mode size d_k as the high word of c * ceil(2^64 / d_k), the
  constant the host computes per launch for the CSR kernel's HCS mode
  indices (Lemire, Kaser and Kurz 2019: exact for every 32-bit c when the
  constant is ceil(2^64 / d) and d < 2^32).
* The second pass of the tensor-core recheck: the largest partial sum of the
  ascending loop over the products, assembled from per-chunk prefix-sum
  extremes offset by an exclusive scan of the chunk totals, the way a group
  of lanes holding consecutive chunks computes it.  Compared with the direct
  running sum.
* The table sort's bucket path: its bucket digit (the 8 bits ending at the
  highest bit on which a table's keys differ), its group digit (the 8 bits
  below) and the placement inside a group by counting, modelled on the host
  and compared with the stable (key, id) order.
"""
import numpy as np
import pytest


def magic(d: int) -> int:
    """The per-mode constant: (2^64 - 1) // d + 1, 0 for d = 1 (the kernel
    takes the quotient as c itself then)."""
    return ((1 << 64) - 1) // d + 1 if d > 1 else 0


def quotient(c: int, M: int) -> int:
    return (M * c) >> 64 if M else c


@pytest.mark.parametrize("d", [1, 2, 3, 7, 10, 12, 13, 17, 23, 71, 100, 200, 256, 1000, 2500, 4096, 65535, 100003,
                               (1 << 31) - 1])
def test_multiply_high_quotient_is_exact(d):
    M = magic(d)
    rng = np.random.default_rng(d)
    cs = [0, 1, d - 1, d, d + 1, 2 * d - 1, (1 << 31) - 1, (1 << 32) - 1]
    cs += [int(v) for v in rng.integers(0, 1 << 32, size=2000, dtype=np.uint64)]
    cs += [k * d + r for k in (1, 5, 1000) for r in (0, d - 1) if k * d + r < (1 << 32)]
    for c in cs:
        q = quotient(c, M)
        assert q == c // d, (c, d)
        assert c - q * d == c % d


def test_constant_is_the_ceiling():
    for d in range(2, 5000):
        M = magic(d)
        assert M == -(-(1 << 64) // d)  # ceil(2^64 / d)


def max_partial_by_scan(products: np.ndarray, per: int, G: int) -> int:
    """Largest |partial sum| of the ascending loop, computed the way the kernel
    does: chunks of `per` products, lane gl of a group of G holding chunk
    c0 + gl in iteration c0 / G."""
    n = len(products)
    nch = n // per
    run = 0
    big = 0
    for c0 in range(0, nch, G):
        T, qmax, qmin = [0] * G, [0] * G, [0] * G
        for gl in range(G):
            c = c0 + gl
            if c >= nch:
                continue
            t, hi, lo = 0, None, None
            for k in range(per):
                t += int(products[c * per + k])
                hi = t if hi is None else max(hi, t)
                lo = t if lo is None else min(lo, t)
            T[gl], qmax[gl], qmin[gl] = t, hi, lo
        incl = np.cumsum(np.array(T, dtype=object))
        for gl in range(G):
            if c0 + gl >= nch:
                continue
            base = run + int(incl[gl]) - T[gl]
            big = max(big, abs(base + qmax[gl]), abs(base + qmin[gl]))
        run += int(incl[G - 1])
    return big


@pytest.mark.parametrize("G,per,d", [(8, 8, 960), (32, 8, 960), (8, 16, 512), (32, 16, 2048), (8, 8, 8), (32, 8, 72)])
def test_partial_sum_scan_equals_running_sum(G, per, d):
    rng = np.random.default_rng(G * 1000 + d)
    for trial in range(20):
        # integer products of mixed signs and magnitudes (up to 2^52)
        mag = rng.integers(0, 1 << 20, size=d) << rng.integers(0, 32, size=d)
        sign = rng.choice([-1, 1], size=d)
        if trial % 4 == 0:
            sign[: d // 2] = 1  # a long same-sign run: the extreme is inside a chunk
        prods = [int(s) * int(m) for s, m in zip(sign, mag)]
        direct = 0
        t = 0
        for p in prods:
            t += p
            direct = max(direct, abs(t))
        assert max_partial_by_scan(np.array(prods, dtype=object), per, G) == direct


# ---- the bucket sort's choice of digits, on the host ----
#
# The table sort's bucket path picks its digits from the bits on which a
# table's keys differ (OR of the keys AND OR of their complements): the
# bucket digit is the 8 bits ending at the highest such bit, the group digit
# the 8 bits below it, and a key's place is its group's start plus the number
# of group members with a smaller key or an equal key earlier in id order.
# The model below makes those choices the way the kernels do and must give
# the stable (key, id) order on key sets that reach each case.

def _varying(keys):
    o1 = np.bitwise_or.reduce(keys)
    o0 = np.bitwise_or.reduce(~keys)
    return int(o1 & o0)


def _msd_shift(v):
    hi = v.bit_length() - 1 if v else 0
    return hi - 7 if hi >= 8 else 0


def _bucket_order(keys):
    """ids of one table in the order the bucket path produces (groups of any
    size are placed by counting here; the kernels send groups above 96 keys to
    the global-memory passes, which give the same stable order)."""
    keys = np.asarray(keys, np.uint64)
    n = keys.size
    msd = _msd_shift(_varying(keys))
    s2 = msd - 8 if msd >= 8 else 0
    ids = np.arange(n)
    bdig = ((keys >> np.uint64(msd)) & np.uint64(255)).astype(np.int64)
    out = []
    for b in range(256):
        members = ids[bdig == b]                 # stable: id order
        if members.size == 0:
            continue
        k = keys[members]
        # every bit at or above msd agrees inside a bucket
        assert np.all((k >> np.uint64(msd)) == (k[0] >> np.uint64(msd)))
        g = ((k >> np.uint64(s2)) & np.uint64(255)).astype(np.int64)
        order = np.argsort(g, kind="stable")     # the counting pass
        k, members, g = k[order], members[order], g[order]
        placed = np.empty_like(members)
        for gv in np.unique(g):
            pos = np.nonzero(g == gv)[0]
            a = pos[0]
            for i in pos:
                r = int(np.sum(k[pos] < k[i])) + int(np.sum((k[pos] == k[i]) & (pos < i)))
                placed[a + r] = members[i]
        out.append(placed)
    return np.concatenate(out)


def _key_sets():
    rng = np.random.default_rng(7)
    u = lambda n: rng.integers(0, 2**64, size=n, dtype=np.uint64)
    yield "uniform", u(3000)
    yield "eleven_bit", rng.integers(0, 2**11, size=3000, dtype=np.uint64)
    yield "three_bit", rng.integers(0, 8, size=500, dtype=np.uint64)
    yield "one_value", np.full(300, np.uint64(0xDEADBEEF12345678))
    yield "bit63_and_low48", (u(2000) & np.uint64((1 << 48) - 1)) | (u(2000) & np.uint64(1 << 63))
    yield "few_values", u(6)[rng.integers(0, 6, size=2000)]
    low = u(3) & np.uint64((1 << 56) - 1)
    yield "top_byte_and_three_low", (rng.integers(0, 256, size=2000, dtype=np.uint64) << np.uint64(56)) | \
        low[rng.integers(0, 3, size=2000)]
    yield "single", u(1)


@pytest.mark.parametrize("name,keys", list(_key_sets()), ids=lambda x: x if isinstance(x, str) else "")
def test_bucket_path_digits_give_the_stable_order(name, keys):
    want = np.lexsort((np.arange(keys.size), keys))   # key, then id
    got = _bucket_order(keys)
    assert np.array_equal(got, want), name


def test_msd_shift_cases():
    assert _msd_shift(0) == 0                # one key value: the pass sorts on bits 0-7
    assert _msd_shift(0b1011) == 0           # fewer than 9 varying bits: one pass suffices
    assert _msd_shift(1 << 8) == 1           # the bucket digit ends at the highest varying bit
    assert _msd_shift((1 << 64) - 1) == 56
    assert _msd_shift((1 << 63) | 1) == 56
