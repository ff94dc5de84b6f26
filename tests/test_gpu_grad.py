"""GPU adjoints (Sec. 2.3) against the FP64 oracle's closed-form gradients on
the same seeded inputs.  Vector cotangents and point gradients: norm-wise
relative 1e-4.  Kernel parameter gradients: every component within 1e-4 of
itself (FP32 recompute of the k x k factors, summed over all points in
FP64)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import TOL, assert_theta, np_, rel_norm, theta_rel, to_gpu

pytestmark = pytest.mark.gpu

CASES = [
    ("uniform", 3000, 8, (1, 1.0, 0.1, 1e-4)),
    # the differentiation workload's kernel at N = 2^12: SE, l = 0.03, nugget 1e-4, k = 32
    ("uniform", 4096, 32, (3, 1.0, 0.03, 1e-4)),
    # the same kernel at k = 16 (one thread per point in the recompute)
    ("uniform", 4096, 16, (3, 1.0, 0.03, 1e-4)),
    ("gaussian", 3000, 16, (1, 1.0, 0.1, 1e-6)),
    # theta_bar of this case is held to 1e-3 (THETA_TOL): its sigma2
    # component is a difference of terms ~20x larger than itself
    ("ldr", 3000, 5, (2, 1.2, 0.1, 1e-3)),
    # 32 < k <= 64: one warp per point, the factor in shared memory
    ("uniform", 3000, 48, (1, 1.0, 0.03, 1e-4)),
    ("gaussian", 3000, 64, (0, 1.0, 0.1, 1e-4)),
]


def _setup(gg, kind, N, k, kern):
    pts = workloads.cloud(kind, N, 60 + k)
    want = oracle.build_graph(pts, k, 64)
    g = gg.build_graph(to_gpu(pts), k, n0=64)
    K = oracle.Kernel(*kern)
    fo = oracle.factor(want["pts_pos"], want["nbr_pos"], k, 64, K)
    f = gg.factor(g, gg.Kernel(*kern))
    return g, f, want, fo, K


def _theta_close(got, want, tol=TOL):
    assert_theta(got, want, tol)


# named cases whose theta_bar is held to 1e-3 instead of 1e-4
THETA_TOL = {("ldr", 3000, 5, (2, 1.2, 0.1, 1e-3)): 1e-3}


def _tol(want, kern, k):
    return TOL


@pytest.mark.parametrize("case", CASES)
def test_nll_gradient(gpu_lib, case):
    kind, N, k, kern = case
    g, f, want, fo, K = _setup(gpu_lib, kind, N, k, kern)
    v = oracle.generate(fo, want["nbr_pos"], k, 64,
                        workloads.white_noise(N, 61).astype(np.float64)).astype(np.float32)
    vbar_or, tb_or = oracle.nll_grad(want, K, v.astype(np.float64))
    vbar, tb = gpu_lib.nll_backward(g, f, to_gpu(v))
    tol = _tol(want, kern, k)
    assert rel_norm(np_(vbar), vbar_or) < tol, rel_norm(np_(vbar), vbar_or)
    _theta_close(np_(tb), tb_or, THETA_TOL.get(case, tol))


@pytest.mark.parametrize("case", CASES)
def test_whiten_vjp(gpu_lib, case):
    kind, N, k, kern = case
    g, f, want, fo, K = _setup(gpu_lib, kind, N, k, kern)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(N).astype(np.float32)
    xibar = rng.standard_normal(N).astype(np.float32)
    xi_or = oracle.whiten(fo, want["nbr_pos"], k, 64, v.astype(np.float64))
    a = oracle.whiten_vjp(fo, want["nbr_pos"], k, 64, v.astype(np.float64), xi_or,
                          xibar.astype(np.float64), 0.7)
    tb_or = oracle.factor_backward(want["pts_pos"], want["nbr_pos"], k, 64, K, a["bbar"], a["bdbar"],
                                   a["sigbar"])
    xi = gpu_lib.whiten(g, f, to_gpu(v))
    vbar, tb = gpu_lib.whiten_backward(g, f, to_gpu(v), xi, to_gpu(xibar), 0.7)
    tol = _tol(want, kern, k)
    assert rel_norm(np_(vbar), a["vbar"]) < tol, rel_norm(np_(vbar), a["vbar"])
    _theta_close(np_(tb), tb_or, THETA_TOL.get(case, tol))


@pytest.mark.parametrize("case", CASES)
def test_generate_vjp(gpu_lib, case):
    kind, N, k, kern = case
    g, f, want, fo, K = _setup(gpu_lib, kind, N, k, kern)
    rng = np.random.default_rng(4)
    xi = rng.standard_normal(N).astype(np.float32)
    vbar = rng.standard_normal(N).astype(np.float32)
    v_or = oracle.generate(fo, want["nbr_pos"], k, 64, xi.astype(np.float64))
    a = oracle.generate_vjp(fo, want["nbr_pos"], k, 64, xi.astype(np.float64), v_or,
                            vbar.astype(np.float64))
    tb_or = oracle.factor_backward(want["pts_pos"], want["nbr_pos"], k, 64, K, a["bbar"], a["bdbar"],
                                   a["sigbar"])
    v = gpu_lib.generate(g, f, to_gpu(xi))
    xibar, tb = gpu_lib.generate_backward(g, f, to_gpu(xi), v, to_gpu(vbar))
    tol = _tol(want, kern, k)
    assert rel_norm(np_(xibar), a["xibar"]) < tol, rel_norm(np_(xibar), a["xibar"])
    _theta_close(np_(tb), tb_or, THETA_TOL.get(case, tol))


def test_thetabar_accumulates(gpu_lib):
    g, f, want, fo, K = _setup(gpu_lib, "uniform", 2000, 8, (1, 1.0, 0.1, 1e-4))
    v = to_gpu(workloads.white_noise(2000, 5))
    _, t1 = gpu_lib.nll_backward(g, f, v)
    t2 = t1.clone()
    gpu_lib.nll_backward(g, f, v, thetabar=t2)
    assert torch.allclose(t2, 2 * t1, rtol=1e-6)


@pytest.mark.parametrize("k", [8, 16, 32])
def test_vector_only_vjps(gpu_lib, k):
    """theta=False passes no thetabar: the per-row factor backward is skipped
    and the vector cotangents are those of the full call (the transposed
    sums are atomic, so equal to rounding)."""
    N = 3000
    g, f, want, fo, K = _setup(gpu_lib, "gaussian", N, k, (1, 1.0, 0.1, 1e-6))
    v = to_gpu(workloads.white_noise(N, 7))
    xi = to_gpu(workloads.white_noise(N, 8))
    cot = to_gpu(workloads.white_noise(N, 9))
    for full, part in [
            (gpu_lib.nll_backward(g, f, v), gpu_lib.nll_backward(g, f, v, theta=False)),
            (gpu_lib.whiten_backward(g, f, v, xi, cot, 0.5),
             gpu_lib.whiten_backward(g, f, v, xi, cot, 0.5, theta=False)),
            (gpu_lib.generate_backward(g, f, xi, v, cot),
             gpu_lib.generate_backward(g, f, xi, v, cot, theta=False))]:
        assert part[1] is None
        assert rel_norm(np_(part[0]), np_(full[0])) < 1e-6


def _max_cond(want, K, k, rows=200):
    """Largest condition number of K_cc over sampled rows (numpy, FP64)."""
    x = want["pts_pos"].astype(np.float64)
    n0 = want["n0"]
    out = 0.0
    for i in np.linspace(n0, want["N"] - 1, rows).astype(int):
        c = want["nbr_pos"][i - n0]
        r = np.sqrt(((x[c][:, None] - x[c][None]) ** 2).sum(-1))
        Kc = np.vectorize(lambda rr: oracle.kappa(K, rr))(r) + K.nugget * np.eye(k)
        out = max(out, np.linalg.cond(Kc))
    return out


def test_ill_conditioned_kernel(gpu_lib):
    """A very smooth kernel (SE, l = 0.3 on a unit-Gaussian cloud of 3000
    points: cond(K_cc) ~1e5): vbar to the stated 1e-4, theta_bar to 1e-3 per
    component (its sigma2 component is a difference of terms ~4000x larger
    than itself)."""
    g, f, want, fo, K = _setup(gpu_lib, "gaussian", 3000, 16, (3, 1.0, 0.3, 1e-4))
    cond = _max_cond(want, K, 16)
    assert cond > 1e4
    v = oracle.generate(fo, want["nbr_pos"], 16, 64,
                        workloads.white_noise(3000, 61).astype(np.float64)).astype(np.float32)
    vbar_or, tb_or = oracle.nll_grad(want, K, v.astype(np.float64))
    vbar, tb = gpu_lib.nll_backward(g, f, to_gpu(v))
    assert rel_norm(np_(vbar), vbar_or) < TOL, (cond, rel_norm(np_(vbar), vbar_or))
    _theta_close(np_(tb), tb_or, 1e-3)


def test_autograd_functions_match_oracle(gpu_lib):
    """torch.autograd over the C-ABI adjoints: d NLL / d(v, theta) and the
    chain generate -> whiten against the oracle's closed forms."""
    from paper_2606_11402_gb300 import autograd as ga
    kind, N, k, kern = CASES[0]
    g, f, want, fo, K = _setup(gpu_lib, kind, N, k, kern)
    theta = torch.tensor([kern[2], kern[1], kern[3]], dtype=torch.float64, requires_grad=True)
    v = oracle.generate(fo, want["nbr_pos"], k, 64,
                        workloads.white_noise(N, 71).astype(np.float64)).astype(np.float32)
    vt = to_gpu(v).requires_grad_(True)
    loss = ga.nll(g, kern[0], theta, vt)
    loss.backward()
    vbar_or, tb_or = oracle.nll_grad(want, K, v.astype(np.float64))
    assert rel_norm(np_(vt.grad), vbar_or) < 1e-4
    _theta_close(theta.grad.numpy(), tb_or)
    # generate then a linear functional: d/dxi = L^T w, d/dtheta vs oracle
    xi = workloads.white_noise(N, 72)
    w = np.random.default_rng(5).standard_normal(N).astype(np.float32)
    theta2 = theta.detach().clone().requires_grad_(True)
    xit = to_gpu(xi).requires_grad_(True)
    out = ga.generate(g, kern[0], theta2, xit)
    (out * to_gpu(w)).sum().backward()
    a = oracle.generate_vjp(fo, want["nbr_pos"], k, 64, xi.astype(np.float64),
                            oracle.generate(fo, want["nbr_pos"], k, 64, xi.astype(np.float64)),
                            w.astype(np.float64))
    tb2 = oracle.factor_backward(want["pts_pos"], want["nbr_pos"], k, 64, K, a["bbar"], a["bdbar"],
                                 a["sigbar"])
    assert rel_norm(np_(xit.grad), a["xibar"]) < 1e-4
    _theta_close(theta2.grad.numpy(), tb2)
    # logdet alone
    theta3 = theta.detach().clone().requires_grad_(True)
    ga.logdet(g, kern[0], theta3).backward()
    z = np.zeros(N)
    a3 = oracle.whiten_vjp(fo, want["nbr_pos"], k, 64, z, z, z, 1.0)
    tb3 = oracle.factor_backward(want["pts_pos"], want["nbr_pos"], k, 64, K, a3["bbar"],
                                 a3["bdbar"], a3["sigbar"])
    _theta_close(theta3.grad.numpy(), tb3)


@pytest.mark.parametrize("k,kern", [(8, (1, 1.0, 0.1, 1e-4)), (32, (3, 1.0, 0.03, 1e-4))])
def test_autograd_nll_fit_equals_nll(gpu_lib, k, kern):
    """nll_fit (value and gradient from one pass) against nll (factor, value,
    then the stored-factor gradient): the value to 1e-12, v's gradient to
    1e-6, theta's to 1e-6 of its largest component; and against the
    oracle's closed form at the stated 1e-4.  A cotangent of 2 scales both."""
    from paper_2606_11402_gb300 import autograd as ga
    N = 3000
    g, f, want, fo, K = _setup(gpu_lib, "uniform", N, k, kern)
    v = oracle.generate(fo, want["nbr_pos"], k, 64,
                        workloads.white_noise(N, 73).astype(np.float64)).astype(np.float32)
    grads = []
    for fn in (ga.nll, ga.nll_fit):
        theta = torch.tensor([kern[2], kern[1], kern[3]], dtype=torch.float64, requires_grad=True)
        vt = to_gpu(v).requires_grad_(True)
        loss = fn(g, kern[0], theta, vt)
        (2.0 * loss).backward()
        grads.append((loss.item(), np_(vt.grad), theta.grad.numpy()))
    (l0, vb0, tb0), (l1, vb1, tb1) = grads
    assert abs(l1 - l0) <= 1e-12 * abs(l0)
    assert rel_norm(vb1, vb0) < 1e-6
    assert np.all(np.abs(tb1 - tb0) <= 1e-6 * np.abs(tb0).max()), (tb1, tb0)
    vbar_or, tb_or = oracle.nll_grad(want, K, v.astype(np.float64))
    assert rel_norm(vb1, 2.0 * vbar_or) < 1e-4
    _theta_close(tb1, 2.0 * tb_or)


@pytest.mark.parametrize("case", CASES)
def test_nll_point_gradient(gpu_lib, case):
    """dNLL/d(points) with the graph held fixed, against the oracle (itself
    pinned by finite differences and by the invariances below); the GPU
    result also sums to zero over the points (translation invariance)."""
    kind, N, k, kern = case
    g, f, want, fo, K = _setup(gpu_lib, kind, N, k, kern)
    v = oracle.generate(fo, want["nbr_pos"], k, 64,
                        workloads.white_noise(N, 63).astype(np.float64)).astype(np.float32)
    pb_or = oracle.nll_grad_points(want, K, v.astype(np.float64))
    pb = np_(gpu_lib.nll_backward_points(g, f, to_gpu(v))).astype(np.float64)
    tol = _tol(want, kern, k)
    assert rel_norm(pb, pb_or) < tol, rel_norm(pb, pb_or)
    assert np.all(np.abs(pb.sum(axis=0)) <= tol * np.abs(pb).sum())
    # scaled cotangent
    pb2 = np_(gpu_lib.nll_backward_points(g, f, to_gpu(v), nllbar=-0.5)).astype(np.float64)
    assert rel_norm(pb2, -0.5 * pb) < 1e-6


def test_autograd_nll_with_points(gpu_lib):
    """torch.autograd through the point-differentiable NLL: gradients with
    respect to v, theta and the [N, 2] points the graph was built from (the
    zero-padded third coordinate is dropped).  The plumbing (order, the
    upstream factor 2, the dropped coordinate) is checked against the direct
    entry points to 1e-6; the values against the oracle to 1e-4 (theta_bar:
    1e-3 per component; its sigma2 component is a difference of terms ~200x
    larger than itself on this cloud)."""
    from paper_2606_11402_gb300 import autograd as ga
    N, k, kern = 2500, 8, (1, 1.0, 0.1, 1e-4)
    pts2 = workloads.uniform_cube(N, 81)[:, :2].copy()
    pts3 = np.concatenate([pts2, np.zeros((N, 1), np.float32)], axis=1)
    want = oracle.build_graph(pts3, k, 64)
    P = to_gpu(pts2).requires_grad_(True)
    g = gpu_lib.build_graph(P.detach(), k, n0=64)
    K = oracle.Kernel(*kern)
    fo = oracle.factor(want["pts_pos"], want["nbr_pos"], k, 64, K)
    v = oracle.generate(fo, want["nbr_pos"], k, 64,
                        workloads.white_noise(N, 82).astype(np.float64)).astype(np.float32)
    theta = torch.tensor([kern[2], kern[1], kern[3]], dtype=torch.float64, requires_grad=True)
    vt = to_gpu(v).requires_grad_(True)
    (2.0 * ga.nll(g, kern[0], theta, vt, P)).backward()
    assert P.grad.shape == (N, 2)
    f = gpu_lib.factor(g, gpu_lib.Kernel(*kern))
    vb, tb = gpu_lib.nll_backward(g, f, to_gpu(v))
    pb = gpu_lib.nll_backward_points(g, f, to_gpu(v))
    assert rel_norm(np_(vt.grad), 2.0 * np_(vb)) < 1e-6
    assert np.allclose(theta.grad.numpy(), 2.0 * np_(tb), rtol=1e-6, atol=0.0)
    assert rel_norm(np_(P.grad), 2.0 * np_(pb)[:, :2]) < 1e-6
    vbar_or, tb_or = oracle.nll_grad(want, K, v.astype(np.float64))
    pb_or = oracle.nll_grad_points(want, K, v.astype(np.float64))
    assert rel_norm(np_(vt.grad), 2.0 * vbar_or) < TOL
    _theta_close(theta.grad.numpy(), 2.0 * tb_or, 1e-3)
    assert rel_norm(np_(P.grad), 2.0 * pb_or[:, :2]) < TOL, rel_norm(np_(P.grad), 2.0 * pb_or[:, :2])
