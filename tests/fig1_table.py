"""The numbers behind Fig. 1 (Sec. 2.2) on synthetic data, from the FP64
oracle alone (CPU; run ``python tests/fig1_table.py``).  Not collected by
pytest; tests/test_oracle_graph.py and tests/test_oracle_factor.py hold the
qualitative checks.

Centre panel -- number of parallel batches (depth levels, the dense first
block counted as one) for N = 10^4 points from a 3-D unit Gaussian, k = 16,
n0 = 50, in four generation orders: the GraphGP order (bit-reversed k-d tree),
the standard k-d tree order (heap order of the same tree), a random order and
the x-sorted order.  The depth recurrence d_i = 1 + max_{j in c(i)} d_j is
applied to each order with its own preceding-kNN lists (brute force, FP64
distances).

Right panel -- accuracy against the number of neighbours k for Matern
nu = 1/2, 3/2, 5/2 with unit variance.  The divergence of the Vecchia
approximation from the truth is KL(N(0, K) || N(0, K~)): with exact
conditionals every row of the whitening operator W = K~^-1/2 (in the sense
K~^-1 = W^T W) satisfies w_i^T K w_i = 1 (sigma_i^2 is exactly the
conditional variance that K assigns), so tr(K~^-1 K) = N and the divergence
reduces to (log det K~ - log det K) / 2, with log det K~ = 2 sum log sigma_i
from the oracle's factor and log det K from a dense FP64 Cholesky.  The
caption's "cutoff rho = 10" is read as the lengthscale rho = 10 mean
nearest-neighbour distances of the cloud (an assumption: the text does not
define rho); a nugget of 1e-6 keeps the dense K positive definite.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402


def levels_for_order(x, perm, k, n0):
    """Depth levels of generating x in the order perm with k-nearest-
    preceding conditioning (brute force, FP64 distances)."""
    y = x[perm].astype(np.float64)
    N = len(perm)
    depth = np.zeros(N, np.int64)
    for j in range(n0, N):
        d = ((y[:j] - y[j]) ** 2).sum(axis=1)
        nb = np.argpartition(d, k - 1)[:k] if j > k else np.arange(j)
        depth[j] = 1 + depth[nb].max()
    return int(depth.max()) + 1


def standard_tree_order(g, N):
    """Heap order of the same k-d tree (children 2h+1, 2h+2)."""
    order, frontier = [], [(0, 0)]
    heap = {}
    while frontier:
        j, h = frontier.pop()
        if j >= N:
            continue
        heap[h] = j
        frontier.append((oracle.left(j), 2 * h + 1))
        frontier.append((oracle.right(j), 2 * h + 2))
    return g["tree_point"][[heap[h] for h in sorted(heap)]]


def batches(N=10_000, k=16, n0=50, seed=26):
    pts = oracle.canonicalise(workloads.unit_gaussian(N, seed))
    g = oracle.build_graph(pts, k, n0)
    out = {"GraphGP (bit-reversed k-d tree)": len(g["level_offsets"]) - 1}
    out["standard k-d tree order"] = levels_for_order(pts, standard_tree_order(g, N), k, n0)
    out["random order"] = levels_for_order(pts, np.random.default_rng(3).permutation(N), k, n0)
    out["x-sorted order"] = levels_for_order(pts, np.argsort(pts[:, 0], kind="stable"), k, n0)
    assert levels_for_order(pts, g["tree_point"], k, n0) == out["GraphGP (bit-reversed k-d tree)"]
    return out


def mean_nn_distance(x):
    x = x.astype(np.float64)
    best = np.full(len(x), np.inf)
    for s in range(0, len(x), 1000):
        d = ((x[s:s + 1000, None, :] - x[None, :, :]) ** 2).sum(-1)
        d[np.arange(d.shape[0]), np.arange(s, s + d.shape[0])] = np.inf
        best[s:s + 1000] = d.min(axis=1)
    return float(np.sqrt(best).mean())


def dense_logdet(x, kern):
    y = x.astype(np.float64)
    K = np.empty((len(y), len(y)))
    for s in range(0, len(y), 1000):
        r = np.sqrt(((y[s:s + 1000, None, :] - y[None, :, :]) ** 2).sum(-1))
        a = r / kern.lengthscale
        if kern.type == 0:
            K[s:s + 1000] = np.exp(-a)
        elif kern.type == 1:
            a = np.sqrt(3.0) * a
            K[s:s + 1000] = (1 + a) * np.exp(-a)
        else:
            a = np.sqrt(5.0) * a
            K[s:s + 1000] = (1 + a + a * a / 3) * np.exp(-a)
    K *= kern.sigma2
    K[np.diag_indices_from(K)] += kern.nugget
    sign, ld = np.linalg.slogdet(K)
    assert sign > 0
    return ld


def kl_table(N=10_000, n0=50, seed=26, ks=(1, 2, 4, 8, 16, 32), rho=10.0, nugget=1e-6):
    pts = oracle.canonicalise(workloads.unit_gaussian(N, seed))
    ell = rho * mean_nn_distance(pts)
    rows = {}
    for nu_name, t in (("1/2", 0), ("3/2", 1), ("5/2", 2)):
        kern = oracle.Kernel(t, 1.0, ell, nugget)
        ld_true = dense_logdet(oracle.canonicalise(pts), kern)
        vals = []
        for k in ks:
            g = oracle.build_graph(pts, k, max(n0, k))
            fac = oracle.factor(g["pts_pos"], g["nbr_pos"], k, g["n0"], kern)
            vals.append(0.5 * (fac["logdet"] - ld_true))
        rows[nu_name] = vals
    return ell, ks, rows


def main():
    b = batches()
    print("| order (N = 10^4 unit Gaussian, k = 16, n0 = 50) | batches |")
    print("|---|---|")
    for name, n in b.items():
        print(f"| {name} | {n} |")
    print()
    ell, ks, rows = kl_table()
    print(f"KL(N(0, K) || N(0, K~)) in nats, N = 10^4 unit Gaussian, n0 = 50, lengthscale {ell:.4f}"
          " (10 mean nearest-neighbour distances), nugget 1e-6")
    print()
    print("| nu | " + " | ".join(f"k = {k}" for k in ks) + " |")
    print("|---|" + "---|" * len(ks))
    for nu, vals in rows.items():
        print(f"| {nu} | " + " | ".join("%.3g" % v for v in vals) + " |")


if __name__ == "__main__":
    main()
