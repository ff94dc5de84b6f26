"""GPU graph construction against the oracle: bit-exact k-d tree, neighbour
lists, depths, graph order and level offsets (Sec. 2.2, 2.3)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import gpu_graph_arrays, to_gpu

pytestmark = pytest.mark.gpu


def _cloud(kind, N, seed):
    rng = np.random.default_rng(seed)
    if kind == "grid":  # many exact ties in coordinates and distances
        return rng.integers(0, 7, size=(N, 3)).astype(np.float32) * np.float32(0.25)
    if kind == "dups":  # every point three times
        base = workloads.uniform_cube((N + 2) // 3, seed)
        return np.concatenate([base, base, base])[:N]
    if kind == "flat":  # one constant axis
        p = workloads.uniform_cube(N, seed)
        p[:, 2] = 0.5
        return p
    if kind == "negzero":
        p = workloads.unit_gaussian(N, seed)
        p[::7, 0] = -0.0
        p[1::7, 0] = 0.0
        return p
    return workloads.cloud(kind, N, seed)


def _compare(gg, pts, k, n0=None, rule=0, knn="brute"):
    N = pts.shape[0]
    want = oracle.build_graph(pts, k, n0, rule=rule, knn=knn)
    g = gg.build_graph(to_gpu(pts), k, n0=want["n0"], split_rule=rule)
    got = gpu_graph_arrays(g)
    assert g.n0 == want["n0"] and g.N == N
    assert np.array_equal(got["tree_point"], want["tree_point"])
    assert np.array_equal(got["split_dim"], want["split_dim"])
    assert np.array_equal(got["inorder"], want["inorder"])
    assert np.array_equal(got["nbr_tree"], want["nbr_tree"])
    assert np.array_equal(got["depth"], want["depth"])
    assert np.array_equal(got["order"], want["order"])
    assert np.array_equal(got["level_offsets"], want["level_offsets"])
    assert np.array_equal(got["nbr_pos"], want["nbr_pos"])
    return g, want


def test_tiny_workload_graph_is_bit_exact(gpu_lib):
    """N=4096 uniform points, k=8 (the small workload)."""
    w = workloads.WORKLOADS["tiny"]
    pts = workloads.uniform_cube(w["N"], w["seed"])
    _compare(gpu_lib, pts, w["k"])


@pytest.mark.parametrize("kind", ["uniform", "gaussian", "ldr", "blobs", "grid", "dups", "flat",
                                  "negzero"])
@pytest.mark.parametrize("k", [1, 5, 16, 32, 33, 64])
def test_graph_bit_exact_clouds(gpu_lib, kind, k):
    # 5003 points: several radix-sort tiles (2048) and sweep chunks plus a tail
    pts = _cloud(kind, 5003, 100 + k)
    _compare(gpu_lib, pts, k, n0=max(k, 64))


@pytest.mark.parametrize("rule", [0, 1])
def test_graph_split_rules(gpu_lib, rule):
    pts = workloads.ldr_cloud(3001, 7)
    _compare(gpu_lib, pts, 8, rule=rule)


@pytest.mark.parametrize("N,k,n0", [(1, 1, 1), (2, 1, 1), (3, 2, 2), (64, 8, 64), (65, 8, 64),
                                    (257, 16, 256), (1000, 32, 32), (2049, 4, 2048),
                                    (64, 64, 64), (65, 64, 64), (700, 48, 48)])
def test_graph_edge_sizes(gpu_lib, N, k, n0):
    pts = workloads.unit_gaussian(N, N)
    _compare(gpu_lib, pts, k, n0=n0)


def test_graph_larger_bit_exact(gpu_lib):
    """A larger cloud through the oracle's exact tree search (itself pinned
    to the brute force)."""
    pts = workloads.unit_gaussian(60_001, 8)
    _compare(gpu_lib, pts, 16, knn="tree")


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("kind", ["gaussian", "grid"])
def test_graph_lower_dimensions(gpu_lib, d, kind):
    """float[N][d] input, d < 3: the same graph as the oracle's on the points
    padded with zero coordinates (the d-dimensional definition)."""
    N, k = 5003, 8
    pts3 = _cloud(kind, N, 70 + d)
    pts_d = np.ascontiguousarray(pts3[:, :d])
    padded = np.zeros((N, 3), np.float32)
    padded[:, :d] = pts_d
    want = oracle.build_graph(padded, k, 64)
    g = gpu_lib.build_graph(to_gpu(pts_d), k, n0=64)
    got = gpu_graph_arrays(g)
    for key in ("tree_point", "split_dim", "nbr_tree", "depth", "order", "level_offsets", "nbr_pos"):
        assert np.array_equal(got[key], want[key]), key
    with pytest.raises(gpu_lib.GraphGPError):  # round-robin splits need d = 3
        gpu_lib.build_graph(to_gpu(pts_d), k, n0=64, split_rule=1)


def test_graph_rejects_bad_input(gpu_lib):
    pts = workloads.uniform_cube(100, 1)
    pts[5, 1] = np.nan
    with pytest.raises(gpu_lib.GraphGPError) as e:
        gpu_lib.build_graph(to_gpu(pts), 8)
    assert e.value.status == gpu_lib.ERR_NAN
    with pytest.raises(gpu_lib.GraphGPError):
        gpu_lib.build_graph(to_gpu(workloads.uniform_cube(100, 1)), 65)
    with pytest.raises(gpu_lib.GraphGPError):
        gpu_lib.build_graph(to_gpu(workloads.uniform_cube(100, 1)), 8, n0=4)


def test_graph_save_load_roundtrip(gpu_lib, tmp_path):
    pts = workloads.uniform_cube(3000, 3)
    g = gpu_lib.build_graph(to_gpu(pts), 8)
    p = str(tmp_path / "g.bin")
    g.save(p)
    h = gpu_lib.graph_load(p)
    a, b = g.export(), h.export()
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x.cpu(), y.cpu())


def test_graph_import_of_oracle_graph(gpu_lib):
    pts = workloads.uniform_cube(2000, 4)
    want = oracle.build_graph(pts, 8)
    g = gpu_lib.graph_import(pts, 8, want["n0"], want["order"], want["nbr_pos"],
                             want["level_offsets"])
    order, nbr, lo = g.export()
    torch.cuda.synchronize()
    assert np.array_equal(order.cpu().numpy(), want["order"])
    assert np.array_equal(nbr.cpu().numpy(), want["nbr_pos"])
    assert np.array_equal(lo.numpy(), want["level_offsets"])
    bad = want["nbr_pos"].copy()
    bad[10, 0] = want["level_offsets"][-1] - 1  # a neighbour in a later level
    with pytest.raises(gpu_lib.GraphGPError):
        gpu_lib.graph_import(pts, 8, want["n0"], want["order"], bad, want["level_offsets"])


def test_kernels_report_sm103(gpu_lib):
    """The device code the library loaded was compiled for sm_103a (GB300)."""
    assert gpu_lib.binary_version() == 103
