"""Pins of the oracle's family sampler (the random functions of Definitions 2-5).

The paper only asks for 2-wise independent h: [d] -> [m], s: [d] -> {+1,-1}
(Definitions 4, 5) and Gaussian r (Definitions 2, 3).  The oracle draws fully
random tables from SplitMix64; these tests pin the generator to its published
outputs and the tables to the distributions the definitions require.
"""
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector(orc):
    lines = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
             if ln.strip() and not ln.startswith("#")]
    seed = int(lines[0][1])
    want = [int(ln[0]) for ln in lines[1:]]
    import ctypes
    st = ctypes.c_uint64(seed)
    got = [int(orc.lib().orc_splitmix_next(ctypes.byref(st))) for _ in want]
    assert got == want


def test_table_streams_distinct(orc):
    a = orc.splitmix_stream(42, 0, 64)
    b = orc.splitmix_stream(42, 1, 64)
    c = orc.splitmix_stream(43, 0, 64)
    assert len(set(a) & set(b)) == 0 and len(set(a) & set(c)) == 0


@pytest.mark.parametrize("m", [4, 12, 16, 64, 256])
def test_cs_bins_uniform_signs_balanced(orc, m):
    d, L = 4096, 64
    f = orc.family("cs_e2lsh", d, m, L, seed=11)
    assert f.bins.min() >= 0 and f.bins.max() < m
    counts = np.bincount(f.bins.ravel(), minlength=m)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4, (chi2, p)
    s = f.signs.ravel().astype(np.int64)
    assert set(np.unique(s)) == {-1, 1}
    n = s.size
    assert abs(s.sum()) < 5 * np.sqrt(n)
    # bin and sign come from disjoint bits of the same draw: independent
    tab = np.zeros((m, 2))
    np.add.at(tab, (f.bins.ravel(), (s > 0).astype(int)), 1)
    chi2, p, _, _ = stats.chi2_contingency(tab)
    assert p > 1e-4


def test_hcs_mode_tables(orc):
    f = orc.family("hcs_e2lsh", 960, 64, 8, dims=[8, 10, 12], mdims=[4, 4, 4], seed=5)
    assert f.bins.shape == (8, 30)
    for t in range(8):
        for k, (h, s) in enumerate(f.mode_tables(t)):
            assert h.min() >= 0 and h.max() < 4
            assert set(np.unique(s)) <= {-1, 1}
    # the b offsets: w * U[0,1)
    assert (f.b >= 0).all() and (f.b < f.w).all()
    assert (f.ka % 2 == 1).all() and (f.kb % 2 == 1).all()


def test_offsets_uniform(orc):
    f = orc.family("cs_e2lsh", 16, 64, 400, w=4.0, seed=3)
    u = (f.b / f.w).ravel()
    assert stats.kstest(u, "uniform").pvalue > 1e-4


def test_dense_gaussian(orc):
    f = orc.family("e2lsh", 64, 16, 40, seed=9)
    g = f.G.astype(np.float64).ravel()
    assert abs(g.mean()) < 5 / np.sqrt(g.size)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / g.size)
    assert stats.kstest(g, "norm").pvalue > 1e-4


def test_family_deterministic(orc):
    a = orc.family("cs_srp", 100, 16, 4, seed=77)
    b = orc.family("cs_srp", 100, 16, 4, seed=77)
    c = orc.family("cs_srp", 100, 16, 4, seed=78)
    assert (a.bins == b.bins).all() and (a.signs == b.signs).all()
    assert not (a.bins == c.bins).all()
    # CS tables are the N = 1 case of the HCS draw order
    h = orc.family("hcs_srp", 100, 16, 4, dims=[100], mdims=[16], seed=77)
    assert (h.bins == a.bins).all() and (h.signs == a.signs).all()
