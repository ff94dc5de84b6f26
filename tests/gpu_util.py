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
