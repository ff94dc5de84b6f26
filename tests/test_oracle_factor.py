"""Pins of the oracle's covariance, factor and sweeps (Sec. 2.1 Eq. 1-2,
Alg. 1, Sec. 3) against textbook routines (LAPACK through numpy, scipy's
Bessel functions) and the exactness statement of Sec. 2.1."""
import numpy as np
import pytest
from scipy.special import gamma, kv

import oracle
import workloads

KERNELS = [oracle.Kernel(t, 1.3, 0.2, 1e-6) for t in (0, 1, 2, 3)]


def _matern_bessel(nu, s2, ell, r):
    """General Matern covariance through the modified Bessel function."""
    if r == 0.0:
        return s2
    z = np.sqrt(2.0 * nu) * r / ell
    return s2 * 2.0 ** (1.0 - nu) / gamma(nu) * z ** nu * kv(nu, z)


@pytest.mark.parametrize("t,nu", [(0, 0.5), (1, 1.5), (2, 2.5)])
def test_matern_closed_forms_equal_bessel_form(t, nu):
    for r in [0.0, 1e-4, 0.01, 0.1, 0.37, 1.0, 3.0]:
        want = _matern_bessel(nu, 1.3, 0.2, r)
        assert oracle.kappa(oracle.Kernel(t, 1.3, 0.2, 0.0), r) == pytest.approx(want, rel=1e-10, abs=1e-300)


def test_sqexp_is_matern_limit():
    """The squared exponential is the nu -> infinity limit of Matern."""
    for r in [0.01, 0.1, 0.3]:
        se = oracle.kappa(oracle.Kernel(3, 1.0, 0.2, 0.0), r)
        assert _matern_bessel(60.0, 1.0, 0.2, r) == pytest.approx(se, rel=2e-2)


@pytest.mark.parametrize("kern", KERNELS)
def test_dkappa_dell_by_central_difference(kern):
    for r in [0.0, 0.03, 0.2, 0.5]:
        h = 1e-6 * kern.lengthscale
        kp = oracle.kappa(kern._replace(lengthscale=kern.lengthscale + h), r)
        km = oracle.kappa(kern._replace(lengthscale=kern.lengthscale - h), r)
        assert oracle.dkappa_dell(kern, r) == pytest.approx((kp - km) / (2 * h), rel=1e-6, abs=1e-9)


def _dense_K(pts, kern):
    x = pts.astype(np.float64)
    r = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    K = np.vectorize(lambda rr: oracle.kappa(kern, rr))(r)
    K[np.diag_indices_from(K)] = oracle.kappa(kern, 0.0) + kern.nugget
    return K


def _implied_L(fac, g, k, n0):
    """L with v = L xi, column by column from generate on unit vectors."""
    N = g["N"]
    L = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        L[:, j] = oracle.generate(fac, g["nbr_pos"], k, n0, e)
    return L


@pytest.mark.parametrize("kern", KERNELS)
def test_dense_block_is_textbook_cholesky(kern):
    """n0 = N: the whole field is the dense initial batch of Alg. 1."""
    N = 256
    pts = oracle.canonicalise(workloads.uniform_cube(N, 31))
    g = oracle.build_graph(pts, 8, n0=N)
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], 8, N, kern)
    K = _dense_K(g["pts_pos"], kern)
    Lnp = np.linalg.cholesky(K)
    assert np.allclose(fac["L0"], Lnp, rtol=0, atol=1e-10 * np.abs(Lnp).max())
    sign, ld = np.linalg.slogdet(K)
    assert sign > 0 and fac["logdet"] == pytest.approx(ld, rel=1e-10)


@pytest.mark.parametrize("kern", [KERNELS[1], KERNELS[3]])
def test_full_conditioning_rows_are_exact(kern):
    """Sec. 2.1: if c(i) holds all preceding points the approximation is exact
    and equals the dense Cholesky factor.  Here n0 = 1 and k = N - 1, so every
    row goes through the per-point conditional path."""
    N = 96
    pts = oracle.canonicalise(workloads.uniform_cube(N, 32))
    g = oracle.build_graph(pts, N - 1, n0=1)
    k = N - 1
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, 1, kern)
    L = _implied_L(fac, g, k, 1)
    K = _dense_K(g["pts_pos"], kern)
    Lnp = np.linalg.cholesky(K)
    assert np.allclose(L, Lnp, rtol=0, atol=1e-10)
    assert fac["logdet"] == pytest.approx(np.linalg.slogdet(K)[1], rel=1e-10)


@pytest.mark.parametrize("kern", KERNELS)
def test_weights_and_sigma_match_linear_solve(kern):
    """Eq. 2: b_i = K_cc^-1 K_ci and sigma_i^2 = K_ii - K_ic b_i, here by a
    general LAPACK solve on every row."""
    N, k = 1500, 8
    g = oracle.build_graph(workloads.unit_gaussian(N, 33), k)
    n0 = g["n0"]
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kern)
    x = g["pts_pos"].astype(np.float64)
    for i in range(n0, N, 7):
        c = g["nbr_pos"][i - n0]
        idx = np.r_[c, i]
        K = _dense_K(x[idx], kern)
        bb = np.linalg.solve(K[:k, :k], K[:k, k])
        s2 = K[k, k] - K[k, :k] @ bb
        assert np.allclose(fac["b"][i - n0], bb, rtol=1e-9, atol=1e-9 * np.abs(bb).max())
        assert fac["sigma"][i] == pytest.approx(np.sqrt(s2), rel=1e-9)


@pytest.mark.parametrize("kern", KERNELS)
def test_alg1_joint_form_equals_weight_form(kern):
    """Alg. 1: L[k+1,1:k] L[1:k,1:k]^-1 v_c + L[k+1,k+1] xi_i equals
    b_i . v_c + sigma_i xi_i."""
    N, k = 2048, 8
    g = oracle.build_graph(workloads.uniform_cube(N, 34), k)
    n0 = g["n0"]
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kern)
    xi = workloads.white_noise(N, 35).astype(np.float64)
    v = oracle.generate(fac, g["nbr_pos"], k, n0, xi)
    va = oracle.generate_alg1(g["pts_pos"], g["nbr_pos"], k, n0, kern, xi)
    assert np.allclose(v, va, rtol=0, atol=1e-11 * np.abs(v).max())


def test_whiten_inverts_generate_and_logdet_of_implied_covariance():
    kern = oracle.Kernel(1, 1.0, 0.1, 1e-6)
    N, k = 400, 8
    g = oracle.build_graph(workloads.uniform_cube(N, 36), k, n0=16)
    n0 = g["n0"]
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kern)
    xi = workloads.white_noise(N, 37).astype(np.float64)
    v = oracle.generate(fac, g["nbr_pos"], k, n0, xi)
    assert np.allclose(oracle.whiten(fac, g["nbr_pos"], k, n0, v), xi, atol=1e-9)
    L = _implied_L(fac, g, k, n0)
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.allclose(np.diag(L), fac["sigma"])
    Kt = L @ L.T
    sign, ld = np.linalg.slogdet(Kt)
    assert sign > 0 and fac["logdet"] == pytest.approx(ld, rel=1e-9)
    # the implied precision (I-B)^T D^-2 (I-B) is sparse: row i of L^-1
    # touches only i and c(i)
    Linv = np.linalg.inv(L)
    for i in range(n0, N):
        nz = set(np.flatnonzero(np.abs(Linv[i]) > 1e-8 * np.abs(Linv[i]).max()))
        assert nz <= set(g["nbr_pos"][i - n0].tolist()) | {i}


def test_kl_to_truth_decreases_with_k():
    """Fig. 1 (right), qualitatively: accuracy improves with the number of
    neighbours.  KL(N(0, K~) || N(0, K)) for k = 2, 4, 8, 16."""
    kern = oracle.Kernel(1, 1.0, 0.15, 1e-6)
    N = 300
    pts = workloads.unit_gaussian(N, 38) * np.float32(0.3)
    kls = []
    for k in (2, 4, 8, 16):
        g = oracle.build_graph(pts, k, n0=k)
        fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, k, kern)
        L = _implied_L(fac, g, k, k)
        Kt = L @ L.T
        K = _dense_K(g["pts_pos"], kern)
        Kinv = np.linalg.inv(K)
        kl = 0.5 * (np.trace(Kinv @ Kt) - N + np.linalg.slogdet(K)[1] - fac["logdet"])
        kls.append(kl)
    assert all(a > b for a, b in zip(kls, kls[1:])), kls
    assert kls[-1] >= -1e-9


def test_not_pd_clamp_counts_duplicate_points():
    """Duplicated points with no nugget make K_cc singular; the pivot floor
    keeps the factor finite and counts the rows (reading of Sec. 2.1)."""
    base = workloads.uniform_cube(300, 39)
    pts = np.concatenate([base, base])
    kern = oracle.Kernel(1, 1.0, 0.2, 0.0)
    g = oracle.build_graph(pts, 8, n0=8)
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], 8, 8, kern)
    assert fac["n_not_pd"] > 0
    assert np.isfinite(fac["b"]).all() and np.isfinite(fac["sigma"]).all()
