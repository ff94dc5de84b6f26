"""The measured configurations at their full sizes, built and factored as the
benchmark builds them (n0 = 256, the same kernels):

* large-dynamic-range cloud, N = 2^20, k = 16: the whole graph bit-exact
  against the oracle's, factor and sweeps against the oracle's FP64 values;
* differentiation workload, N = 2^22, k = 32: the k-d tree bit-exact against
  the oracle's, sampled neighbour lists and factor rows from the oracle, the
  depth recurrence and graph order checked everywhere, adjoint identity;
* headline workload, N = 2^26, k = 16, and scale workload, N = 2^29: checks
  that hold at any size (tree invariants, depth recurrence, order), sampled
  neighbour lists by exact brute force, sampled factor rows from the oracle
  on those independently found neighbours, the sweeps' round trip and the
  log-determinant's reduction."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from fullsize import check_depth_and_order, check_tree, inorder_rank_of, inorder_ranks, knn_sample
from gpu_util import LDR_RESCUE, LDR_TOL, gpu_graph_arrays, np_, rel_norm, sigma_rel, to_gpu

pytestmark = pytest.mark.gpu

N0 = 256


def _samples(N, n0, extra, seed):
    rng = np.random.default_rng(seed)
    js = [n0, n0 + 1, n0 + 17, min(N - 1, 4 * n0), N // 3, N // 2, N - 2, N - 1]
    js += list(rng.integers(n0, N, size=extra))
    return np.unique(np.array(js, np.int64))


def _check_rows(pts, tp, js, nbrs_tree, b_rows, sig_rows, kern, tol):
    """b and sigma of the GPU at the sampled tree indices js against the
    oracle's FP64 conditional on the neighbour lists nbrs_tree (tree indices,
    found independently of the GPU): b norm-wise over the sampled rows and
    sigma element-wise, each within tol."""
    K = oracle.Kernel(*kern)
    idx = tp[js]
    nb_in = np.where(nbrs_tree >= 0, tp[np.maximum(nbrs_tree, 0)], -1).astype(np.int32)
    b_or, s_or = oracle.factor_rows(pts, idx, nb_in, K)
    eb, es = rel_norm(b_rows, b_or), sigma_rel(sig_rows, s_or)
    print(f"sampled rows ({len(js)}): b {eb:.2e}, sigma {es:.2e}")
    assert eb < tol and es < tol, (eb, es, tol)


def _positions(order):
    pos_of_input = np.empty(len(order), np.int64)
    pos_of_input[np.asarray(order, np.int64)] = np.arange(len(order))
    return pos_of_input


def _sweep_properties(gg, g, f, N, seed, sigma):
    """whiten(generate(xi)) = xi, and logdet = 2 sum log sigma (FP64)."""
    xi = to_gpu(workloads.white_noise(N, seed))
    v = gg.generate(g, f, xi)
    back = gg.whiten(g, f, v)
    torch.cuda.synchronize()
    rt = float(torch.linalg.vector_norm((back - xi).double()) / torch.linalg.vector_norm(xi.double()))
    assert rt < 1e-4, rt
    del back
    own = 2.0 * float(torch.log(sigma.double()).sum())
    ld = float(gg.logdet(f).item())
    assert abs(ld - own) <= 1e-9 * abs(own)
    st, _ = gg.sync_status(g, f)
    assert st >= 0
    return xi, v


def test_ldr_workload_full_oracle(gpu_lib):
    """N = 2^20 large-dynamic-range cloud, k = 16, Matern-3/2 l = 0.05 without
    nugget: the complete oracle graph, factor and sweeps."""
    w = workloads.WORKLOADS["ldr"]
    N, k, kern = w["N"], w["k"], w["kernel"]
    pts = workloads.ldr_cloud(N, w["seed"])
    want = oracle.build_graph(pts, k, N0, knn="tree")
    g = gpu_lib.build_graph(to_gpu(pts), k, n0=N0)
    got = gpu_graph_arrays(g)
    for key in ("tree_point", "split_dim", "inorder", "nbr_tree", "depth", "order",
                "level_offsets", "nbr_pos"):
        assert np.array_equal(got[key], want[key]), key
    K = oracle.Kernel(*kern)
    fo = oracle.factor(want["pts_pos"], want["nbr_pos"], k, N0, K)
    f = gpu_lib.factor(g, gpu_lib.Kernel(*kern, rescue_tol=LDR_RESCUE))
    b, sigma, _ = (np_(t) for t in f.export())
    tol = LDR_TOL
    print(f"ldr 2^20: b rel {rel_norm(b, fo['b']):.2e}, sigma max rel "
          f"{sigma_rel(sigma, fo['sigma']):.2e}")
    assert rel_norm(b, fo["b"]) < tol
    assert sigma_rel(sigma, fo["sigma"]) < tol
    xi = workloads.white_noise(N, w["xi_seed"])
    v_or = oracle.generate(fo, want["nbr_pos"], k, N0, xi.astype(np.float64))
    v = np_(gpu_lib.generate(g, f, to_gpu(xi)))
    print(f"ldr 2^20: v rel {rel_norm(v, v_or):.2e}")
    assert rel_norm(v, v_or) < tol
    v_in = v_or.astype(np.float32)
    xi_or = oracle.whiten(fo, want["nbr_pos"], k, N0, v_in.astype(np.float64))
    xi_g = np_(gpu_lib.whiten(g, f, to_gpu(v_in)))
    print(f"ldr 2^20: xi rel {rel_norm(xi_g, xi_or):.2e}")
    assert rel_norm(xi_g, xi_or) < tol
    ld = np_(gpu_lib.logdet(f))[0]
    print(f"ldr 2^20: logdet {ld:.6f} oracle {fo['logdet']:.6f}")
    assert abs(ld - fo["logdet"]) <= 2.0 * np.sum(np.abs(sigma / fo["sigma"] - 1.0)) * 1.01 + 1e-9 * abs(fo["logdet"])


def test_diff_workload_full_size(gpu_lib):
    """N = 2^22 uniform cube, k = 32, squared exponential l = 0.03, nugget 1e-4."""
    w = workloads.WORKLOADS["diff"]
    N, k, kern = w["N"], w["k"], w["kernel"]
    pts = oracle.canonicalise(workloads.uniform_cube(N, w["seed"]))
    tp, sd, io = oracle.tree_build(pts)
    g = gpu_lib.build_graph(to_gpu(pts), k, n0=N0)
    got = gpu_graph_arrays(g)
    assert np.array_equal(got["tree_point"], tp)
    assert np.array_equal(got["split_dim"], sd)
    assert np.array_equal(got["inorder"], io)
    check_depth_and_order(got["nbr_tree"], got["depth"], got["inorder"], got["tree_point"],
                          got["order"], got["level_offsets"], got["nbr_pos"], N0)
    js = _samples(N, N0, 24, 1)
    nb_or = oracle.knn_brute_some(pts, tp, js, k)
    assert np.array_equal(got["nbr_tree"][js - N0], nb_or)
    f = gpu_lib.factor(g, gpu_lib.Kernel(*kern))
    b, sigma, _ = f.export()
    pos = _positions(got["order"])[tp[js]]
    pos_t = torch.as_tensor(pos, device="cuda")
    _check_rows(pts, tp, js, nb_or, np_(b[pos_t - N0]), np_(sigma[pos_t]), kern, 1e-3)
    del b
    xi, v = _sweep_properties(gpu_lib, g, f, N, w["xi_seed"], sigma)
    # adjoint identity at full size: <L xi, u> = <xi, L^T u>
    u = to_gpu(workloads.white_noise(N, 77))
    xibar, _ = gpu_lib.generate_backward(g, f, xi, v, u)
    lhs = float(torch.dot(v.double(), u.double()))
    rhs = float(torch.dot(xi.double(), xibar.double()))
    scale = float(torch.linalg.vector_norm(v.double()) * torch.linalg.vector_norm(u.double()))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)


def _generate_rows(b_rows, sig_rows, nbr_rows, pos, v, xi):
    """v_i = b_i . v_c(i) + sigma_i xi_i at the sampled positions, in FP64 from
    the sweep's output and the stored factor rows."""
    vc = np_(v[torch.as_tensor(nbr_rows.astype(np.int64), device="cuda")]).astype(np.float64)
    pt = torch.as_tensor(pos, device="cuda")
    want = (b_rows.astype(np.float64) * vc).sum(1) + sig_rows * np_(xi[pt]).astype(np.float64)
    got = np_(v[pt]).astype(np.float64)
    scale = np.abs(b_rows * vc).sum(1) + np.abs(sig_rows * np_(xi[pt]))
    assert np.all(np.abs(got - want) <= 1e-5 * scale + 1e-30), np.max(np.abs(got - want) / scale)


def test_metric_workload_full_size(gpu_lib):
    """N = 2^26 unit-Gaussian cloud, k = 16, Matern-3/2 l = 0.1, nugget 1e-6:
    the benchmark's workload and build."""
    w = workloads.WORKLOADS["metric"]
    N, k, kern = w["N"], w["k"], w["kernel"]
    pts = oracle.canonicalise(workloads.unit_gaussian(N, w["seed"]))
    g = gpu_lib.build_graph(to_gpu(pts), k, n0=N0)
    torch.cuda.empty_cache()
    got = gpu_graph_arrays(g)
    tp = got["tree_point"].astype(np.int64)
    check_tree(pts, tp, got["split_dim"])
    assert np.array_equal(got["inorder"], inorder_ranks(N))
    check_depth_and_order(got["nbr_tree"], got["depth"], got["inorder"], tp, got["order"],
                          got["level_offsets"], got["nbr_pos"], N0)
    X = pts[tp]
    js = _samples(N, N0, 8, 2)
    nb = np.stack([knn_sample(X, int(j), k) for j in js])
    assert np.array_equal(got["nbr_tree"][js - N0], nb)
    pos = _positions(got["order"])[tp[js]]
    nbr_rows = got["nbr_pos"][pos - N0]
    del got, X
    f = gpu_lib.factor(g, gpu_lib.Kernel(*kern))
    b, sigma, _ = f.export()
    pos_t = torch.as_tensor(pos, device="cuda")
    b_rows, sig_rows = np_(b[pos_t - N0]), np_(sigma[pos_t])
    del b
    torch.cuda.empty_cache()
    _check_rows(pts, tp, js, nb, b_rows, sig_rows, kern, 1e-3)
    xi, v = _sweep_properties(gpu_lib, g, f, N, w["xi_seed"], sigma)
    _generate_rows(b_rows, sig_rows, nbr_rows, pos, v, xi)


def test_scale_workload_full_size(gpu_lib):
    """N = 2^29 clustered cloud (10^4 blobs + 10 % background), k = 16,
    Matern-3/2 l = 0.02, nugget 1e-6: tree invariants and in-order ranks on
    sampled nodes, graph order everywhere, sampled neighbour lists, depths
    and factor rows, sweep round trip and log-determinant."""
    w = workloads.WORKLOADS["scale"]
    N, k, kern = w["N"], w["k"], w["kernel"]
    pts = oracle.canonicalise(workloads.blobs(N, w["seed"]))
    pts_d = to_gpu(pts)
    g = gpu_lib.build_graph(pts_d, k, n0=N0)
    del pts_d
    torch.cuda.empty_cache()
    tp_d, sd_d, io_d, dp_d, nt_d = g.export_tree()
    rng = np.random.default_rng(3)
    js = np.unique(np.r_[N0, N0 + 1, 5000, rng.integers(N0, 1 << 16, 2), N - 1].astype(np.int64))
    nt_rows = np_(nt_d[torch.as_tensor(js - N0, device="cuda")]).astype(np.int64)
    del nt_d
    torch.cuda.empty_cache()
    tp, sd, io, dp = (np_(t) for t in (tp_d, sd_d, io_d, dp_d))
    del tp_d, sd_d, io_d, dp_d
    nodes = np.unique(np.r_[np.arange(1 << 16), rng.integers(0, N, 1 << 18)]).astype(np.int64)
    check_tree(pts, tp, sd, nodes=nodes, check_split_rule=False)
    assert np.array_equal(io[nodes], inorder_rank_of(nodes, N))
    assert np.all(dp[js] == 1 + dp[nt_rows].max(axis=1))
    X = pts[tp]
    nb = np.stack([knn_sample(X, int(j), k) for j in js])
    assert np.array_equal(nt_rows, nb)
    del X
    order_d, nbr_d, lo = g.export()
    order = np_(order_d).astype(np.int64)
    pos = _positions(order)[tp[js]]
    nbr_rows = np_(nbr_d[torch.as_tensor(pos - N0, device="cuda")])
    del order_d, nbr_d
    torch.cuda.empty_cache()
    # graph order: levels by depth, in-order ranks increasing inside a level
    tree_of_input = np.empty(N, np.int64)
    tree_of_input[tp] = np.arange(N)
    t_of_pos = tree_of_input[order]
    d_pos = dp[t_of_pos].astype(np.int64)
    assert np.array_equal(lo.numpy(), np.r_[0, np.cumsum(np.bincount(dp))])
    step = np.diff(d_pos * N + io[t_of_pos].astype(np.int64))
    assert np.all(step > 0)
    del tree_of_input, t_of_pos, d_pos, step, order
    f = gpu_lib.factor(g, gpu_lib.Kernel(*kern))
    b, sigma, _ = f.export()
    pos_t = torch.as_tensor(pos, device="cuda")
    b_rows, sig_rows = np_(b[pos_t - N0]), np_(sigma[pos_t])
    del b
    torch.cuda.empty_cache()
    _check_rows(pts, tp, js, nb, b_rows, sig_rows, kern, 1e-2)
    xi, v = _sweep_properties(gpu_lib, g, f, N, w["xi_seed"], sigma)
    _generate_rows(b_rows, sig_rows, nbr_rows, pos, v, xi)
