"""Pins of the oracle's adjoints (Sec. 2.3: forward and backward derivatives)
by central finite differences in FP64, adjoint dot-product identities and the
closed form of the variance derivative."""
import numpy as np
import pytest

import oracle
import workloads

KERNS = {
    "matern32": oracle.Kernel(1, 1.0, 0.12, 1e-4),
    "sqexp": oracle.Kernel(3, 0.8, 0.09, 1e-4),
    "matern12": oracle.Kernel(0, 1.2, 0.15, 1e-3),
    "matern52": oracle.Kernel(2, 1.0, 0.1, 1e-4),
}


def _graph(N=600, k=8, n0=24, seed=41):
    return oracle.build_graph(workloads.uniform_cube(N, seed), k, n0=n0)


def _nll(g, kern, v):
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], g["k"], g["n0"], kern)
    return oracle.nll(fac, g["nbr_pos"], g["k"], g["n0"], v)


def _theta_fd(fun, kern, rel=1e-4):
    """Central differences with a relative step per parameter."""
    out = []
    for name in ("lengthscale", "sigma2", "nugget"):
        x = getattr(kern, name)
        h = rel * abs(x)
        fp = fun(kern._replace(**{name: x + h}))
        fm = fun(kern._replace(**{name: x - h}))
        out.append((fp - fm) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("name", sorted(KERNS))
def test_nll_gradient_by_finite_differences(name):
    kern = KERNS[name]
    g = _graph()
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], g["k"], g["n0"], kern)
    v = oracle.generate(fac, g["nbr_pos"], g["k"], g["n0"],
                        workloads.white_noise(g["N"], 42).astype(np.float64))
    vbar, tb = oracle.nll_grad(g, kern, v)
    fd = _theta_fd(lambda kk: _nll(g, kk, v), kern)
    assert np.allclose(tb, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    # directional derivative in v
    w = np.random.default_rng(0).standard_normal(g["N"])
    h = 1e-5
    dfd = (_nll(g, kern, v + h * w) - _nll(g, kern, v - h * w)) / (2 * h)
    assert vbar @ w == pytest.approx(dfd, rel=1e-6)


def test_generate_gradient_by_finite_differences():
    """theta-gradient of <generate(xi; theta), w> and its xi-gradient."""
    kern = KERNS["matern32"]
    g = _graph(seed=43)
    k, n0, N = g["k"], g["n0"], g["N"]
    xi = workloads.white_noise(N, 44).astype(np.float64)
    w = np.random.default_rng(1).standard_normal(N)

    def f(kk):
        fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kk)
        return oracle.generate(fac, g["nbr_pos"], k, n0, xi) @ w

    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kern)
    v = oracle.generate(fac, g["nbr_pos"], k, n0, xi)
    a = oracle.generate_vjp(fac, g["nbr_pos"], k, n0, xi, v, w)
    tb = oracle.factor_backward(g["pts_pos"], g["nbr_pos"], k, n0, kern, a["bbar"], a["bdbar"], a["sigbar"])
    fd = _theta_fd(f, kern)
    assert np.allclose(tb, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    # generate is linear in xi: xibar = L^T w
    z = np.random.default_rng(2).standard_normal(N)
    assert a["xibar"] @ z == pytest.approx(oracle.generate(fac, g["nbr_pos"], k, n0, z) @ w, rel=1e-10)


def test_whiten_vjp_is_transpose_of_whiten():
    """<L^-1 v, w> = <v, L^-T w>: the whiten VJP with logdetbar = 0."""
    kern = KERNS["sqexp"]
    g = _graph(seed=45)
    k, n0, N = g["k"], g["n0"], g["N"]
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kern)
    rng = np.random.default_rng(3)
    v, w = rng.standard_normal(N), rng.standard_normal(N)
    xi = oracle.whiten(fac, g["nbr_pos"], k, n0, v)
    a = oracle.whiten_vjp(fac, g["nbr_pos"], k, n0, v, xi, w, 0.0)
    assert a["vbar"] @ v == pytest.approx(xi @ w, rel=1e-10)


def test_logdet_gradient_by_finite_differences():
    kern = KERNS["matern52"]
    g = _graph(seed=46)
    k, n0, N = g["k"], g["n0"], g["N"]
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kern)
    a = oracle.whiten_vjp(fac, g["nbr_pos"], k, n0, np.zeros(N), np.zeros(N), np.zeros(N), 1.0)
    tb = oracle.factor_backward(g["pts_pos"], g["nbr_pos"], k, n0, kern, a["bbar"], a["bdbar"], a["sigbar"])
    fd = _theta_fd(lambda kk: oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kk)["logdet"], kern)
    assert np.allclose(tb, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_variance_gradient_closed_form():
    """With no nugget K scales with sigma2, so with xi1 the field whitened at
    sigma2 = 1: dNLL/dsigma2 = (N - xi1.xi1 / sigma2) / (2 sigma2)."""
    s2 = 1.7
    kern = oracle.Kernel(1, s2, 0.12, 0.0)
    g = _graph(seed=47)
    k, n0, N = g["k"], g["n0"], g["N"]
    v = np.random.default_rng(4).standard_normal(N)
    fac1 = oracle.factor(g["pts_pos"], g["nbr_pos"], k, n0, kern._replace(sigma2=1.0))
    xi1 = oracle.whiten(fac1, g["nbr_pos"], k, n0, v)
    _, tb = oracle.nll_grad(g, kern, v)
    assert tb[1] == pytest.approx((N - xi1 @ xi1 / s2) / (2 * s2), rel=1e-9)


# ---- gradient with respect to the point coordinates (graph held fixed) ------

def _nll_at(g, kern, v, pts_pos):
    fac = oracle.factor(pts_pos, g["nbr_pos"], g["k"], g["n0"], kern)
    return oracle.nll(fac, g["nbr_pos"], g["k"], g["n0"], v)


@pytest.mark.parametrize("name", sorted(KERNS))
def test_point_gradient_by_finite_differences(name):
    """Central differences on single coordinates.  The step 2^-12 is exact in
    FP32 for coordinates in [0, 1), so the perturbed points are exactly the
    intended ones; the graph (order and neighbour lists) stays as built."""
    kern = KERNS[name]
    g = _graph(N=300, k=6, n0=20, seed=47)
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], g["k"], g["n0"], kern)
    v = oracle.generate(fac, g["nbr_pos"], g["k"], g["n0"],
                        workloads.white_noise(g["N"], 48).astype(np.float64))
    xb = oracle.nll_grad_points(g, kern, v)  # input order
    order = np.asarray(g["order"])
    rng = np.random.default_rng(5)
    h = 2.0 ** -12
    # positions from the dense block, the first sparse rows and the last ones
    for pos in (3, 17, 21, 150, g["N"] - 1):
        for d in rng.choice(3, size=2, replace=False):
            pp, pm = g["pts_pos"].copy(), g["pts_pos"].copy()
            pp[pos, d] += np.float32(h)
            pm[pos, d] -= np.float32(h)
            fd = (_nll_at(g, kern, v, pp) - _nll_at(g, kern, v, pm)) / (2 * h)
            got = xb[order[pos], d]
            assert got == pytest.approx(fd, rel=2e-3, abs=1e-5 * np.abs(xb).max()), (pos, d)


@pytest.mark.parametrize("name", ["matern32", "sqexp", "matern52"])
def test_point_gradient_invariances(name):
    """A stationary kernel makes the NLL invariant under a common shift of the
    points (sum of the point gradients = 0), and homogeneous of degree 0 in
    (points, lengthscale) jointly, so sum_p x_p . xbar_p = -l dNLL/dl with the
    lengthscale derivative of the (separately pinned) parameter gradient."""
    kern = KERNS[name]
    g = _graph(N=400, k=8, n0=24, seed=49)
    fac = oracle.factor(g["pts_pos"], g["nbr_pos"], g["k"], g["n0"], kern)
    v = oracle.generate(fac, g["nbr_pos"], g["k"], g["n0"],
                        workloads.white_noise(g["N"], 50).astype(np.float64))
    xb = oracle.nll_grad_points(g, kern, v)
    scale = np.abs(xb).sum()
    assert np.all(np.abs(xb.sum(axis=0)) <= 1e-10 * scale)
    _, tb = oracle.nll_grad(g, kern, v)
    pts = np.asarray(g["pts"], np.float64)  # input order, like xb
    euler = float((pts * xb).sum())
    assert euler == pytest.approx(-kern.lengthscale * tb[0], rel=1e-8)
