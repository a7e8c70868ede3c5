"""Statistical pins of the oracle against the identities and collision
probabilities the paper derives.

Exact over the random family (any d):
* E[CS(p)_l] = 0 and Var[CS(p)_l] = ||p||^2 / m (Theorem 13's proof, Sec. 4.1);
  the same for vec(HCS(p))_l (Theorem 20's proof, Sec. 4.2).
* zero covariance between different bins (Theorem 15's proof).
* E[CS(u)_l CS(v)_l] = <u, v> / m (Theorem 26), the same for HCS (Theorem 32).
* dense E2LSH collision probability p(R) (the integral after Definition 2) and
  dense SRP collision probability 1 - theta/pi (after Definition 3).

Asymptotic in d (checked at large d with a finite-d allowance):
* CS-E2LSH / HCS-E2LSH per-coordinate collision p(R) and all-m collision
  p(R)^m (Theorems 17, 23);
* CS-SRP / HCS-SRP per-bit collision 1 - theta/pi (Theorems 29, 35).

Each Monte-Carlo sample is one independent table of one family; the tolerance
is 5 standard errors of the per-table means (plus the stated finite-d
allowance for the asymptotic results).
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats


def p_e2lsh(R, w):
    """Closed form of p(R) = int_0^w (1/R) f(t/R) (1 - t/w) dt, f = density of |N(0,1)|."""
    c = w / R
    return 1 - 2 * stats.norm.cdf(-c) - 2 / (math.sqrt(2 * math.pi) * c) * (1 - math.exp(-c * c / 2))


@pytest.mark.parametrize("R,w", [(0.5, 4.0), (1.0, 4.0), (2.0, 4.0), (4.0, 4.0), (3.0, 1.0)])
def test_pR_closed_form_matches_paper_integral(R, w):
    f = lambda u: 2 * stats.norm.pdf(u)
    val, _ = integrate.quad(lambda t: (1 / R) * f(t / R) * (1 - t / w), 0, w)
    assert abs(val - p_e2lsh(R, w)) < 1e-10


def _moment_check(Y, want, tol_sd=5.0):
    """Y: [T] per-table samples; check |mean - want| <= tol_sd * se."""
    se = Y.std(ddof=1) / math.sqrt(len(Y))
    assert abs(Y.mean() - want) <= tol_sd * se + 1e-12, (Y.mean(), want, se)


@pytest.mark.parametrize("kind,dims,mdims", [("cs_e2lsh", None, None), ("hcs_e2lsh", [6, 10], [4, 4]),
                                             ("hcs_e2lsh", [3, 4, 5], [2, 4, 2])])
def test_sketch_moments(orc, kind, dims, mdims):
    d, m, T = 60, 16, 20000
    f = orc.family(kind, d, m, T, seed=21, dims=dims, mdims=mdims)
    rng = np.random.default_rng(21)
    u = rng.standard_normal(d).astype(np.float32)
    v = (0.6 * u + 0.8 * rng.standard_normal(d)).astype(np.float32)
    st, y, _, _ = orc.hash_dense(f, np.stack([u, v]), want_codes=False, want_keys=False)
    yu, yv = y[0], y[1]                     # [T, m]
    u64, v64 = u.astype(np.float64), v.astype(np.float64)
    nu2 = float(u64 @ u64)
    for l in (0, 5, m - 1):
        _moment_check(yu[:, l], 0.0)
        _moment_check(yu[:, l] ** 2, nu2 / m)
        _moment_check(yu[:, l] * yv[:, l], float(u64 @ v64) / m)
    _moment_check(yu[:, 0] * yu[:, 1], 0.0)
    _moment_check(yu[:, 3] * yu[:, 12], 0.0)


def _pair(d, R, rng):
    p = rng.standard_normal(d)
    delta = rng.standard_normal(d)
    delta *= R / np.linalg.norm(delta)
    return np.stack([p, p + delta]).astype(np.float32)


def _collision_rates(orc, f, X):
    st, y, codes, keys = orc.hash_dense(f, X, want_y=False)
    eq = codes[0] == codes[1]               # [L, m]
    per_table = eq.mean(axis=1)
    all_equal = eq.all(axis=1)
    return per_table, all_equal


@pytest.mark.parametrize("R", [0.5, 1.5, 3.0])
def test_dense_e2lsh_collision_exact(orc, R):
    d, m, L, w = 32, 16, 4000, 4.0
    f = orc.family("e2lsh", d, m, L, w=w, seed=31)
    rng = np.random.default_rng(31)
    X = _pair(d, R, rng)
    Rr = float(np.linalg.norm(X[0].astype(np.float64) - X[1].astype(np.float64)))
    per_table, _ = _collision_rates(orc, f, X)
    _moment_check(per_table, p_e2lsh(Rr, w))


@pytest.mark.parametrize("cosine", [0.9, 0.5, 0.0, -0.5])
def test_dense_srp_collision_exact(orc, cosine):
    d, m, L = 32, 16, 4000
    f = orc.family("srp", d, m, L, seed=32)
    rng = np.random.default_rng(32)
    a = rng.standard_normal(d)
    b = rng.standard_normal(d)
    b -= (a @ b) / (a @ a) * a
    u = a / np.linalg.norm(a)
    v = cosine * u + math.sqrt(1 - cosine ** 2) * b / np.linalg.norm(b)
    X = np.stack([u, v]).astype(np.float32)
    c = float(X[0].astype(np.float64) @ X[1].astype(np.float64)
              / np.linalg.norm(X[0].astype(np.float64)) / np.linalg.norm(X[1].astype(np.float64)))
    per_table, _ = _collision_rates(orc, f, X)
    _moment_check(per_table, 1 - math.acos(c) / math.pi)


# Asymptotic results: large d, spread (Gaussian) vectors; an allowance on top of
# 5 standard errors for the finite-d deviation from normality.  For a count
# sketch at d = 8000, m = 16 each bin sums ~500 terms and 0.01 suffices.  The
# HCS results (Theorems 20, 23, 35) need sqrt(m) N^(4/5) = o(d^((3N-8)/(10N))),
# which converges very slowly (d^(1/30) for N = 3, no guarantee at all for
# N = 2); at d = 8000 the bins are a scale mixture of normals with the exact
# variance ||p||^2/m but heavier tails, which raises collisions by ~0.03, so the
# HCS allowance is 0.05 (an empirical check of the direction of the result,
# not of its limit).
ASYM = 0.01
ASYM_HCS = 0.05


@pytest.mark.parametrize("kind,dims,mdims", [("cs_e2lsh", None, None), ("hcs_e2lsh", [20, 20, 20], [2, 2, 4]),
                                             ("hcs_e2lsh", [80, 100], [4, 4])])
@pytest.mark.parametrize("R", [1.0, 3.0])
def test_sketch_e2lsh_collision_asymptotic(orc, kind, dims, mdims, R):
    d, m, L, w = 8000, 16, 1500, 4.0
    f = orc.family(kind, d, m, L, w=w, seed=41, dims=dims, mdims=mdims)
    rng = np.random.default_rng(41)
    X = _pair(d, R, rng)
    Rr = float(np.linalg.norm(X[0].astype(np.float64) - X[1].astype(np.float64)))
    per_table, _ = _collision_rates(orc, f, X)
    se = per_table.std(ddof=1) / math.sqrt(L)
    allow = ASYM_HCS if kind.startswith("hcs") else ASYM
    assert abs(per_table.mean() - p_e2lsh(Rr, w)) <= 5 * se + allow


def test_cs_e2lsh_all_m_collision(orc):
    # Theorem 17: all m coordinates collide with probability p(R)^m
    d, m, L, w, R = 8000, 4, 4000, 4.0, 1.0
    f = orc.family("cs_e2lsh", d, m, L, w=w, seed=43)
    X = _pair(d, R, np.random.default_rng(43))
    Rr = float(np.linalg.norm(X[0].astype(np.float64) - X[1].astype(np.float64)))
    _, all_eq = _collision_rates(orc, f, X)
    want = p_e2lsh(Rr, w) ** m
    se = math.sqrt(want * (1 - want) / L)
    assert abs(all_eq.mean() - want) <= 5 * se + ASYM


@pytest.mark.parametrize("kind,dims,mdims", [("cs_srp", None, None), ("hcs_srp", [20, 20, 20], [2, 2, 4]),
                                             ("hcs_srp", [80, 100], [4, 4])])
@pytest.mark.parametrize("cosine", [0.8, 0.2])
def test_sketch_srp_collision_asymptotic(orc, kind, dims, mdims, cosine):
    d, m, L = 8000, 16, 1500
    f = orc.family(kind, d, m, L, seed=44, dims=dims, mdims=mdims)
    rng = np.random.default_rng(44)
    a = rng.standard_normal(d)
    b = rng.standard_normal(d)
    b -= (a @ b) / (a @ a) * a
    u = a / np.linalg.norm(a)
    v = cosine * u + math.sqrt(1 - cosine ** 2) * b / np.linalg.norm(b)
    X = np.stack([u, v]).astype(np.float32)
    c = float(X[0].astype(np.float64) @ X[1].astype(np.float64)
              / np.linalg.norm(X[0].astype(np.float64)) / np.linalg.norm(X[1].astype(np.float64)))
    per_table, _ = _collision_rates(orc, f, X)
    se = per_table.std(ddof=1) / math.sqrt(L)
    allow = ASYM_HCS if kind.startswith("hcs") else ASYM
    assert abs(per_table.mean() - (1 - math.acos(c) / math.pi)) <= 5 * se + allow


def test_collision_monotone_in_distance(orc):
    # The LSH property (Definition 1): nearer pairs collide more often.
    d, m, L, w = 4000, 16, 600, 4.0
    f = orc.family("cs_e2lsh", d, m, L, w=w, seed=45)
    rng = np.random.default_rng(45)
    rates = []
    for R in (0.5, 2.0, 8.0):
        per_table, _ = _collision_rates(orc, f, _pair(d, R, rng))
        rates.append(per_table.mean())
    assert rates[0] > rates[1] > rates[2]
