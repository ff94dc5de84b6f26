"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import torch


def to_gpu(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def np_(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def gpu_graph_arrays(g):
    """Everything the GPU graph build produced, as numpy arrays."""
    order, nbr, lo = g.export()
    tp, sd, io, dp, nt = g.export_tree()
    torch.cuda.synchronize()
    return dict(order=np_(order), nbr_pos=np_(nbr), level_offsets=lo.numpy(),
                tree_point=np_(tp), split_dim=np_(sd), inorder=np_(io), depth=np_(dp),
                nbr_tree=np_(nt))


def rel_norm(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def _kappa_np(kern, r):
    t, s2, ell, _ = kern
    if t == 0:
        return s2 * np.exp(-r / ell)
    if t == 1:
        a = np.sqrt(3.0) * r / ell
        return s2 * (1 + a) * np.exp(-a)
    if t == 2:
        a = np.sqrt(5.0) * r / ell
        return s2 * (1 + a + a * a / 3) * np.exp(-a)
    return s2 * np.exp(-r * r / (2 * ell * ell))


def fp32_tolerance(want, kern, rows=300, base=1e-4):
    """Tolerance for FP32 results on a given graph and kernel.

    Evaluating the covariance in FP32 perturbs every entry of K_cc by about
    2^-24 relative, so the conditional weights move by up to cond(K_cc) 2^-24
    and sigma^2 = K_ii - K_ic b loses another factor K_ii / sigma^2 to
    cancellation.  Returns (tol_vectors, tol_sigma): the stated 1e-4 when the
    conditioning allows it, else 8 x the bound over sampled rows."""
    x = want["pts_pos"].astype(np.float64)
    n0, k = want["n0"], want["k"]
    worst_b, worst_s = 0.0, 0.0
    N = want["N"]
    if N <= n0:
        return base, base
    for i in np.unique(np.linspace(n0, N - 1, rows).astype(int)):
        c = want["nbr_pos"][i - n0]
        idx = np.r_[c, i]
        r = np.sqrt(((x[idx][:, None] - x[idx][None]) ** 2).sum(-1))
        K = _kappa_np(kern, r) + kern[3] * np.eye(k + 1)
        Kc = K[:k, :k]
        cond = np.linalg.cond(Kc)
        b = np.linalg.solve(Kc, K[:k, k])
        s2 = K[k, k] - K[k, :k] @ b
        worst_b = max(worst_b, cond)
        worst_s = max(worst_s, cond * K[k, k] / max(s2, 1e-300))
    eps = 2.0 ** -24
    return max(base, 8 * worst_b * eps), max(base, 8 * worst_s * eps)


def row_tolerance(xc, xq, kern, base=1e-4):
    """fp32_tolerance's bound for one conditional: neighbours xc [k, 3], point
    xq [3]."""
    x = np.vstack([np.asarray(xc, np.float64), np.asarray(xq, np.float64)[None]])
    k = len(xc)
    r = np.sqrt(((x[:, None] - x[None]) ** 2).sum(-1))
    K = _kappa_np(kern, r) + kern[3] * np.eye(k + 1)
    Kc = K[:k, :k]
    cond = np.linalg.cond(Kc)
    b = np.linalg.solve(Kc, K[:k, k])
    s2 = K[k, k] - K[k, :k] @ b
    eps = 2.0 ** -24
    return max(base, 8 * cond * eps), max(base, 8 * cond * K[k, k] / max(s2, 1e-300) * eps)
