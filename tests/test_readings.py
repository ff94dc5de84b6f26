"""CPU pins of two readings the FP32 factor is built on (no GPU, no oracle):

* the increment (variogram) form of the Vecchia conditional (Sec. 2.1 Eq. 2
  rewritten around the nearest neighbour c0) is the same conditional as the
  covariance form: on random rows, in FP64, both give the same b and sigma^2;
* the polynomial tables of variogram_poly.cuh reproduce the functions they
  were fitted to (checked against mpmath at 40 digits) within FP32 rounding,
  and those functions give the variogram of each kernel without
  cancellation.

A wrong sign, index or term in either form, or a corrupted coefficient,
fails these tests."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
POLY = os.path.join(ROOT, "paper_2606_11402_gb300", "csrc", "variogram_poly.cuh")


def kappa(t, r, s2, ell):
    """Matern nu = 1/2, 3/2, 5/2 and the squared exponential (no nugget)."""
    a = np.asarray(r, np.float64) / ell
    if t == 0:
        return s2 * np.exp(-a)
    if t == 1:
        a = np.sqrt(3.0) * a
        return s2 * (1.0 + a) * np.exp(-a)
    if t == 2:
        a = np.sqrt(5.0) * a
        return s2 * (1.0 + a + a * a / 3.0) * np.exp(-a)
    return s2 * np.exp(-0.5 * a * a)


def dist(x, y):
    return np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(-1))


def covariance_form(X, xq, t, s2, ell, nug):
    k = len(X)
    Kcc = kappa(t, dist(X, X), s2, ell) + nug * np.eye(k)
    kci = kappa(t, np.sqrt(((X - xq) ** 2).sum(-1)), s2, ell)
    b = np.linalg.solve(Kcc, kci)
    return b, s2 + nug - kci @ b


def increment_form(X, xq, t, s2, ell, nug, mutate=None):
    """The system of the increments u_a = v_ca - v_c0 (a >= 1) and w = v_i -
    v_c0 beside v_c0, written with gamma(r) = kappa(0) - kappa(r).  `mutate`
    plants one mistake (for the sensitivity test)."""
    k = len(X)

    def gam(r):
        return s2 - kappa(t, r, s2, ell)

    G = gam(dist(X, X))
    g_i = gam(np.sqrt(((X - xq) ** 2).sum(-1)))
    M = np.empty((k, k))
    m = np.empty(k)
    M[0, 0] = s2 + nug
    m[0] = -(g_i[0] + nug) if mutate != "m0_sign" else g_i[0] + nug
    for a in range(1, k):
        M[a, 0] = M[0, a] = -(G[a, 0] + nug)
        m[a] = G[a, 0] + g_i[0] - g_i[a] + nug
        for c in range(1, k):
            off_nug = nug if mutate != "offdiag_nugget" or a == c else 0.0
            M[a, c] = G[a, 0] + G[c, 0] - G[a, c] + off_nug + nug * (a == c)
    beta = np.linalg.solve(M, m)
    b = beta.copy()
    b[0] = 1.0 + beta[0] - beta[1:].sum()
    var_w = 2.0 * (g_i[0] + nug)
    return b, var_w - m @ beta


@pytest.mark.parametrize("t", [0, 1, 2, 3])
@pytest.mark.parametrize("k", [1, 2, 5, 16, 32])
def test_increment_form_is_the_same_conditional(t, k):
    rng = np.random.default_rng(100 * t + k)
    ell = 0.3
    for _ in range(20):
        X = rng.uniform(0.0, 1.0, (k, 3))
        xq = rng.uniform(0.0, 1.0, 3)
        # nearest neighbour first, as the graph stores the rows
        X = X[np.argsort(((X - xq) ** 2).sum(-1))]
        for nug in (1e-4, 1e-2):
            b1, s1 = covariance_form(X, xq, t, 1.3, ell, nug)
            b2, s2_ = increment_form(X, xq, t, 1.3, ell, nug)
            scale = max(1.0, np.abs(b1).max())
            assert np.abs(b1 - b2).max() <= 1e-7 * scale, (b1, b2)
            assert abs(s1 - s2_) <= 1e-7 * max(s1, 1e-6), (s1, s2_)


@pytest.mark.parametrize("mutate", ["m0_sign", "offdiag_nugget"])
def test_increment_form_comparison_catches_a_wrong_term(mutate):
    """The comparison above is sensitive: flipping the sign of m_0, or
    dropping the nugget from the off-diagonal increments, breaks it."""
    rng = np.random.default_rng(7)
    X = rng.uniform(0.0, 1.0, (8, 3))
    xq = rng.uniform(0.0, 1.0, 3)
    X = X[np.argsort(((X - xq) ** 2).sum(-1))]
    b1, s1 = covariance_form(X, xq, 1, 1.0, 0.3, 1e-2)
    b2, s2_ = increment_form(X, xq, 1, 1.0, 0.3, 1e-2)
    assert np.abs(b1 - b2).max() < 1e-9 and abs(s1 - s2_) < 1e-9
    b3, s3 = increment_form(X, xq, 1, 1.0, 0.3, 1e-2, mutate)
    assert np.abs(b1 - b3).max() > 1e-4 or abs(s1 - s3) > 1e-4 * s1


def _tables():
    text = open(POLY).read()
    out = {}
    for m in re.finditer(r"// (.+?): degree (\d+) on \[([-0-9.e]+), ([-0-9.e]+)\].*?\n"
                         r"__device__ __forceinline__ float (\w+)\(float x\) \{\n"
                         r"\s*constexpr float c\[\d+\] = \{([^}]*)\};", text):
        coeffs = [np.float32(float(c.strip().rstrip("f"))) for c in m.group(6).split(",")]
        out[m.group(5)] = (float(m.group(3)), float(m.group(4)), int(m.group(2)), coeffs)
    return out


def _horner_fma32(cs, x):
    """FP32 Horner with fused multiply-add, as the device code evaluates it
    (the FP64 product of two FP32 values is exact)."""
    x = np.float32(x)
    h = cs[-1]
    for c in reversed(cs[:-1]):
        h = np.float32(np.float64(h) * np.float64(x) + np.float64(c))
    return h


def test_polynomial_tables_match_their_functions():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    funcs = {
        "poly_m32": lambda a: (mp.exp(a) - 1 - a) / a ** 2 if a else mp.mpf(1) / 2,
        "poly_m52": lambda a: (mp.exp(a) - 1 - a - a ** 2 / 3) / a ** 2 if a else mp.mpf(1) / 6,
        "poly_exp1": lambda u: (1 - mp.exp(-u)) / u if u else mp.mpf(1),
    }
    tables = _tables()
    assert set(tables) == set(funcs)
    for name, (lo, hi, deg, cs) in tables.items():
        assert len(cs) == deg + 1
        worst = 0.0
        for x in np.linspace(lo, hi, 2001):
            want = funcs[name](mp.mpf(float(np.float32(x))))
            got = _horner_fma32(cs, x)
            worst = max(worst, abs(float((mp.mpf(float(got)) - want) / want)))
        assert worst < 3e-7, (name, worst)


@pytest.mark.parametrize("t", [0, 1, 2, 3])
def test_variogram_from_the_tables(t):
    """gamma / s2 = 1 - kappa / s2 through the tabulated functions, below the
    switch points: Matern-3/2 a^2 e^-a phi(a) (a < 1), Matern-5/2
    a^2 e^-a phi(a) (a < 2), SE and Matern-1/2 u psi(u) with u = a^2 / 2
    resp. a (u < 1/2); against expm1 in FP64."""
    tables = _tables()
    for r in np.linspace(1e-4, 0.45, 400):
        if t == 1:
            a = np.sqrt(3.0) * r
            got = a * a * np.exp(-a) * np.float64(_horner_fma32(tables["poly_m32"][3], a))
            want = -np.expm1(-a) - a * np.exp(-a)
        elif t == 2:
            a = np.sqrt(5.0) * r
            got = a * a * np.exp(-a) * np.float64(_horner_fma32(tables["poly_m52"][3], a))
            want = -np.expm1(-a) - (a + a * a / 3.0) * np.exp(-a)
        else:
            u = r if t == 0 else 0.5 * r * r
            got = u * np.float64(_horner_fma32(tables["poly_exp1"][3], u))
            want = -np.expm1(-u)
        assert abs(got - want) <= 5e-7 * abs(want), (t, r, got, want)
