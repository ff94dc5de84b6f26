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


# Tolerances against the FP64 oracle.  TOL is the stated one for FP32
# fields: norm-wise relative for vectors (b, L0, v, xi, vbar, xibar, point
# gradients), element-wise relative for sigma, and relative per component
# for the FP64-accumulated kernel-parameter gradient theta_bar.  It is
# asserted on every configured kernel.  LDR_TOL is the bound asserted on the
# large-dynamic-range cloud without nugget (conditionals with condition
# numbers up to ~1e11, 20 % of them floored).
TOL = 1e-4
LDR_TOL = 1e-3
# rescue threshold the nugget-free large-dynamic-range tests factor with
# (graphgp_kernel.rescue_tol): at the default 2^-7 one conditional in 10^6
# keeps a sigma error of 1.7e-3
LDR_RESCUE = 2.0 ** -10


def sigma_rel(s, ref):
    """Largest element-wise relative error of sigma."""
    s = np.asarray(s, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(s / ref - 1.0)))


def theta_rel(got, want):
    """Relative error of every component of theta_bar."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return np.abs(got - want) / np.abs(want)


def assert_theta(got, want, tol=TOL):
    r = theta_rel(got, want)
    assert np.all(r <= tol), (r, got, want)
