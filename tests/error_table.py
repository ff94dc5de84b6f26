"""Measured error of every output of the GPU path against the FP64 oracle, on
the configured workloads, printed as a Markdown table (run on a GPU:
``python tests/error_table.py``).  Not collected by pytest; the asserted
bounds live in the test files.

* tiny workload (N = 4096 uniform, k = 8, Matern-3/2 l = 0.1, nugget 1e-6),
* differentiation kernel at N = 2^12 (uniform, k = 32, SE l = 0.03,
  nugget 1e-4),
* large-dynamic-range workload at full size (N = 2^20, k = 16, Matern-3/2
  l = 0.05, no nugget), against the complete oracle, at the default rescue
  threshold and at 2^-10,
* headline workload (N = 2^26 unit Gaussian, k = 16, Matern-3/2 l = 0.1,
  nugget 1e-6): sampled factor rows against the oracle's conditional on the
  GPU's neighbour lists (themselves checked against brute force in
  test_gpu_fullsize.py).

Vectors: norm-wise relative error; sigma: largest element-wise relative
error; theta_bar: relative error per component (lengthscale, sigma2, nugget);
scalars: relative error."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import paper_2606_11402_gb300 as gg  # noqa: E402
import workloads  # noqa: E402
from gpu_util import np_, rel_norm, sigma_rel, theta_rel, to_gpu  # noqa: E402


def full(pts, k, kern, n0=None, knn="brute", points=True, rescue_tol=0.0):
    out = {}
    want = oracle.build_graph(pts, k, n0, knn=knn)
    g = gg.build_graph(to_gpu(pts), k, n0=want["n0"])
    order, nbr, _ = g.export()
    assert np.array_equal(np_(order), want["order"]) and np.array_equal(np_(nbr), want["nbr_pos"])
    K = oracle.Kernel(*kern)
    fo = oracle.factor(want["pts_pos"], want["nbr_pos"], k, want["n0"], K)
    f = gg.factor(g, gg.Kernel(*kern, rescue_tol=rescue_tol))
    b, sigma, L0 = (np_(t) for t in f.export())
    out["b"] = rel_norm(b, fo["b"])
    out["sigma"] = sigma_rel(sigma, fo["sigma"])
    out["L0"] = rel_norm(L0, fo["L0"])
    N, n0 = g.N, g.n0
    xi = workloads.white_noise(N, 1)
    v_or = oracle.generate(fo, want["nbr_pos"], k, n0, xi.astype(np.float64))
    out["v = generate(xi)"] = rel_norm(np_(gg.generate(g, f, to_gpu(xi))), v_or)
    v_in = v_or.astype(np.float32)
    xi_or = oracle.whiten(fo, want["nbr_pos"], k, n0, v_in.astype(np.float64))
    out["xi = whiten(v)"] = rel_norm(np_(gg.whiten(g, f, to_gpu(v_in))), xi_or)
    out["logdet"] = abs(np_(gg.logdet(f))[0] - fo["logdet"]) / abs(fo["logdet"])
    nll_or = oracle.nll(fo, want["nbr_pos"], k, n0, v_in.astype(np.float64))
    out["NLL"] = abs(np_(gg.nll(g, f, to_gpu(v_in)))[0] - nll_or) / abs(nll_or)
    vbar_or, tb_or = oracle.nll_grad(want, K, v_in.astype(np.float64))
    vbar, tb = gg.nll_backward(g, f, to_gpu(v_in))
    out["vbar (NLL)"] = rel_norm(np_(vbar), vbar_or)
    out["theta_bar (NLL)"] = theta_rel(np_(tb), tb_or)
    nf, vbf, tbf = gg.nll_grad_fused(g, gg.Kernel(*kern, rescue_tol=rescue_tol), to_gpu(v_in))
    out["NLL (fused value and gradient)"] = abs(np_(nf)[0] - nll_or) / abs(nll_or)
    out["vbar (fused value and gradient)"] = rel_norm(np_(vbf), vbar_or)
    out["theta_bar (fused value and gradient)"] = theta_rel(np_(tbf), tb_or)
    w = np.random.default_rng(4).standard_normal(N).astype(np.float32)
    a = oracle.generate_vjp(fo, want["nbr_pos"], k, n0, xi.astype(np.float64), v_or,
                            w.astype(np.float64))
    tg_or = oracle.factor_backward(want["pts_pos"], want["nbr_pos"], k, n0, K, a["bbar"],
                                   a["bdbar"], a["sigbar"])
    xib, tg = gg.generate_backward(g, f, to_gpu(xi), to_gpu(v_or.astype(np.float32)), to_gpu(w))
    out["xibar (generate VJP)"] = rel_norm(np_(xib), a["xibar"])
    out["theta_bar (generate VJP)"] = theta_rel(np_(tg), tg_or)
    if points:
        pb_or = oracle.nll_grad_points(want, K, v_in.astype(np.float64))
        out["point gradients (NLL)"] = rel_norm(np_(gg.nll_backward_points(g, f, to_gpu(v_in))), pb_or)
    return out


def sampled(pts, k, kern, nsamp=3000):
    g = gg.build_graph(to_gpu(pts), k, n0=256)
    order, nbr, _ = g.export()
    order = np_(order)
    rows = np.sort(np.random.default_rng(0).choice(len(pts) - 256, nsamp, replace=False)) + 256
    nb = np_(nbr[torch.as_tensor(rows - 256, device="cuda")])
    b_or, s_or = oracle.factor_rows(pts, order[rows], order[nb].astype(np.int32), oracle.Kernel(*kern))
    f = gg.factor(g, gg.Kernel(*kern))
    b, sigma, _ = f.export()
    rt = torch.as_tensor(rows, device="cuda")
    out = {"b": rel_norm(np_(b[rt - 256]), b_or), "sigma": sigma_rel(np_(sigma[rt]), s_or)}
    xi = to_gpu(workloads.white_noise(len(pts), 7))
    back = gg.whiten(g, f, gg.generate(g, f, xi))
    out["whiten(generate(xi)) = xi"] = float(torch.linalg.vector_norm((back - xi).double())
                                             / torch.linalg.vector_norm(xi.double()))
    return out


def fmt(x):
    if isinstance(x, np.ndarray):
        return " / ".join("%.1e" % v for v in x)
    return "%.1e" % x


def main():
    gg.load()
    cols = [
        ("tiny, N=4096, k=8", lambda: full(workloads.uniform_cube(4096, 0), 8, (1, 1.0, 0.1, 1e-6))),
        ("differentiation kernel, N=2^12, k=32",
         lambda: full(workloads.uniform_cube(4096, 4), 32, (3, 1.0, 0.03, 1e-4))),
        ("large dynamic range, N=2^20, k=16",
         lambda: full(workloads.ldr_cloud(1 << 20, 2), 16, (1, 1.0, 0.05, 0.0), 256, "tree", False)),
        ("the same, rescue_tol 2^-10",
         lambda: full(workloads.ldr_cloud(1 << 20, 2), 16, (1, 1.0, 0.05, 0.0), 256, "tree", False,
                      2.0 ** -10)),
        ("headline, N=2^26, k=16 (3000 sampled rows)",
         lambda: sampled(workloads.unit_gaussian(1 << 26, 6), 16, (1, 1.0, 0.1, 1e-6))),
    ]
    res = [(name, fn()) for name, fn in cols]
    keys = []
    for _, r in res:
        keys += [k for k in r if k not in keys]
    print("| output | " + " | ".join(n for n, _ in res) + " |")
    print("|---|" + "---|" * len(res))
    for key in keys:
        print(f"| {key} | " + " | ".join(fmt(r[key]) if key in r else "-" for _, r in res) + " |")


if __name__ == "__main__":
    main()
