"""GPU adjoints (Sec. 2.3) against the FP64 oracle's closed-form gradients on
the same seeded inputs.  Vector cotangents: norm-wise relative 1e-4.  Kernel
parameter gradients: every component within 2e-3 of the largest one (FP32
recompute of the k x k factors, summed over all points in FP64)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import np_, rel_norm, to_gpu

pytestmark = pytest.mark.gpu

CASES = [
    ("uniform", 3000, 8, (1, 1.0, 0.1, 1e-4)),
    ("gaussian", 3000, 16, (3, 1.0, 0.3, 1e-4)),
    ("uniform", 2500, 32, (3, 1.0, 0.08, 1e-4)),
    ("ldr", 3000, 5, (2, 1.2, 0.1, 1e-3)),
]


def _setup(gg, kind, N, k, kern):
    pts = workloads.cloud(kind, N, 60 + k)
    want = oracle.build_graph(pts, k, 64)
    g = gg.build_graph(to_gpu(pts), k, n0=64)
    K = oracle.Kernel(*kern)
    fo = oracle.factor(want["pts_pos"], want["nbr_pos"], k, 64, K)
    f = gg.factor(g, gg.Kernel(*kern))
    return g, f, want, fo, K


def _theta_close(got, want):
    scale = np.max(np.abs(want))
    assert np.all(np.abs(got - want) <= 2e-3 * scale), (got, want)


@pytest.mark.parametrize("case", CASES)
def test_nll_gradient(gpu_lib, case):
    kind, N, k, kern = case
    g, f, want, fo, K = _setup(gpu_lib, kind, N, k, kern)
    v = oracle.generate(fo, want["nbr_pos"], k, 64,
                        workloads.white_noise(N, 61).astype(np.float64)).astype(np.float32)
    vbar_or, tb_or = oracle.nll_grad(want, K, v.astype(np.float64))
    vbar, tb = gpu_lib.nll_backward(g, f, to_gpu(v))
    assert rel_norm(np_(vbar), vbar_or) < 1e-4
    _theta_close(np_(tb), tb_or)


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
    assert rel_norm(np_(vbar), a["vbar"]) < 1e-4
    _theta_close(np_(tb), tb_or)


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
    assert rel_norm(np_(xibar), a["xibar"]) < 1e-4
    _theta_close(np_(tb), tb_or)


def test_thetabar_accumulates(gpu_lib):
    g, f, want, fo, K = _setup(gpu_lib, "uniform", 2000, 8, (1, 1.0, 0.1, 1e-4))
    v = to_gpu(workloads.white_noise(2000, 5))
    _, t1 = gpu_lib.nll_backward(g, f, v)
    t2 = t1.clone()
    gpu_lib.nll_backward(g, f, v, thetabar=t2)
    assert torch.allclose(t2, 2 * t1, rtol=1e-6)
