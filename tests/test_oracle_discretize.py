"""Pins of the oracle's discretisation (Definitions 2, 3, 12, 19, 25, 31) on
hand-picked values whose results follow from the formulas by hand.

E2LSH family: code = floor((scale * y + b) / w), scale = sqrt(m) for the CS/HCS
variants (Definitions 12, 19) and 1 for dense E2LSH (Definition 2); floor is
the mathematical floor (toward minus infinity).  SRP family: 1 iff y > 0.
"""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("y,scale,b,w,want", [
    (1.5, 2.0, 1.0, 4.0, 1),                        # (3 + 1) / 4 = 1 exactly
    (math.nextafter(1.5, 0.0), 2.0, 1.0, 4.0, 0),   # just below the edge
    (math.nextafter(1.5, 2.0), 2.0, 1.0, 4.0, 1),
    (0.0, 2.0, 1.0, 4.0, 0),                        # b / w = 0.25
    (-0.0, 2.0, 3.99, 4.0, 0),
    (-1.0, 2.0, 1.0, 4.0, -1),                      # -0.25 -> -1 (toward -inf)
    (-0.5, 2.0, 1.0, 4.0, 0),                       # (-1 + 1)/4 = 0 exactly
    (-2.5, 2.0, 1.0, 4.0, -1),                      # -4/4 = -1 exactly
    (-2.5000000001, 2.0, 1.0, 4.0, -2),
    (10.0, 1.0, 2.0, 4.0, 3),                       # dense: (10 + 2)/4 = 3
    (7.0, 4.0, 0.0, 0.5, 56),                       # m = 16: 28 / 0.5
])
def test_e2lsh_edges(orc, y, scale, b, w, want):
    code, err = orc.e2lsh_code(y, scale, b, w)
    assert err == 0
    assert code == want


def test_e2lsh_overflow_flag(orc):
    code, err = orc.e2lsh_code(1e12, 1.0, 0.0, 1.0)
    assert err == 1
    code, err = orc.e2lsh_code(-1e12, 1.0, 0.0, 1.0)
    assert err == 1
    code, err = orc.e2lsh_code(2147483647.0, 1.0, 0.0, 1.0)
    assert err == 0 and code == 2147483647
    code, err = orc.e2lsh_code(-2147483648.0, 1.0, 0.0, 1.0)
    assert err == 0 and code == -2147483648


@pytest.mark.parametrize("y,want", [(0.0, 0), (-0.0, 0), (5e-324, 1), (-5e-324, 0), (1.0, 1),
                                    (-1.0, 0), (float("inf"), 1)])
def test_srp_sign(orc, y, want):
    assert orc.srp_bit(y) == want


def test_sqrt_scale_is_ieee(orc):
    # scale sqrt(m) for m not a square: the code uses the correctly rounded sqrt
    m = 12
    for y in np.linspace(-3, 3, 101):
        code, _ = orc.e2lsh_code(y, math.sqrt(m), 0.7, 4.0)
        assert code == math.floor((math.sqrt(m) * y + 0.7) / 4.0)


def test_empty_bin_codes(orc):
    # a CS bin with no coordinate is exactly 0: SRP bit 0, E2LSH floor(b / w)
    d, m = 3, 64  # d << m leaves most bins empty
    f = orc.family("cs_e2lsh", d, m, 1, seed=1)
    X = np.ones((1, d), np.float32)
    st, y, codes, keys = orc.hash_dense(f, X)
    empty = np.setdiff1d(np.arange(m), f.bins[0])
    assert len(empty) > 0
    assert (y[0, 0, empty] == 0).all()
    assert np.array_equal(codes[0, 0, empty], np.floor(f.b[0, empty] / f.w).astype(np.int32))
    fs = orc.family("cs_srp", d, m, 1, seed=1)
    st, y, codes, keys = orc.hash_dense(fs, X)
    assert (codes[0, 0, empty] == 0).all()


def test_nonfinite_input_status(orc):
    f = orc.family("cs_e2lsh", 8, 4, 1, seed=1)
    X = np.ones((2, 8), np.float32)
    X[1, 3] = np.nan
    st, *_ = orc.hash_dense(f, X)
    assert st & 2
